// gsm_arith.cuh -- arithmetic of the three precisions of the FFT passes.
//
//   F64  : IEEE double.
//   F32  : IEEE single.
//   DF64 : double-float ("FP32x2"): a value is hi + lo with two floats,
//          about 48 significand bits, computed with FP32 instructions only.
//          Additions use the error-free two-sum of Knuth; products use the
//          FMA-based exact product (Dekker 1971, "A floating-point technique
//          for extending the available precision"; Hida, Li, Bailey 2001,
//          double-double).  Tables (twiddles, multiplier) are split from FP64
//          into normalised pairs, |lo| <= ulp(hi)/2; the results of sums and
//          products within a stage are left unnormalised ("pair arithmetic",
//          M. Lange and S. M. Rump, ACM TOMS 46 (2020)): the closing fast
//          two-sum of double-word arithmetic is omitted, so |lo| may exceed
//          ulp(hi)/2, until the value is stored (DF64::st renormalises).
//          The error of each operation stays bounded relative
//          to |a| + |b| (sums) or |a||b| (products with a normalised factor:
//          every product of the passes has a table value, twiddle or
//          multiplier, as one factor), which is what normwise FFT error
//          bounds use.
//
// Every kernel is written once against this interface:
//   real  R          scalar type
//   cx<R>            complex in registers
//   Pol::scplx       complex as stored in shared/global memory
//   Pol::tw_t        twiddle-table entry, Pol::mult_t multiplier entry,
//   Pol::io_t        element type of rho and u
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gsm {

struct df {
    float hi, lo;
};

template <class R>
struct cx {
    R re, im;
};

// ------------------------------------------------------------------ double
__device__ __forceinline__ double radd(double a, double b) { return a + b; }
__device__ __forceinline__ double rsub(double a, double b) { return a - b; }
__device__ __forceinline__ double rneg(double a) { return -a; }
__device__ __forceinline__ double rmul(double a, double b) { return a * b; }
__device__ __forceinline__ double rmulk(double a, double k) { return a * k; }

// ------------------------------------------------------------------ float
__device__ __forceinline__ float radd(float a, float b) { return a + b; }
__device__ __forceinline__ float rsub(float a, float b) { return a - b; }
__device__ __forceinline__ float rneg(float a) { return -a; }
__device__ __forceinline__ float rmul(float a, float b) { return a * b; }
__device__ __forceinline__ float rmulk(float a, double k) { return a * (float)k; }

// ------------------------------------------------------------------ double-float
// s + e == a + b exactly (Knuth two-sum, six additions).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// s + e == a + b exactly when the exponent of a is at least that of b
// (Dekker's fast two-sum, three additions).  Renormalising a pair (hi, lo)
// of the pair arithmetic: |lo| < |hi| except after a cancellation, and then
// s is still a + b rounded and the error of s + e is below u |lo|, well under
// the pair's own error bound, which is relative to the operands before the
// cancellation.
__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}
__device__ __forceinline__ df radd(df a, df b)
{
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    return df{s, __fadd_rn(e, __fadd_rn(a.lo, b.lo))};
}
__device__ __forceinline__ df rneg(df a) { return df{-a.hi, -a.lo}; }
__device__ __forceinline__ df rsub(df a, df b) { return radd(a, rneg(b)); }
// product: p + e == a.hi * b.hi exactly, then the cross terms
__device__ __forceinline__ df rmul(df a, df b)
{
    float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return df{p, e};
}
// split a double constant into hi + lo floats (folds at compile time)
__host__ __device__ __forceinline__ df df_from_double(double k)
{
    float h = (float)k;
    float l = (float)(k - (double)h);
    return df{h, l};
}
__device__ __forceinline__ df rmulk(df a, double k) { return rmul(a, df_from_double(k)); }
__device__ __forceinline__ double df_to_double(df a) { return (double)a.hi + (double)a.lo; }

// ------------------------------------------------------------------ complex
template <class R>
__device__ __forceinline__ cx<R> cadd(cx<R> a, cx<R> b) { return {radd(a.re, b.re), radd(a.im, b.im)}; }
template <class R>
__device__ __forceinline__ cx<R> csub(cx<R> a, cx<R> b) { return {rsub(a.re, b.re), rsub(a.im, b.im)}; }
// multiply by -i (forward) or +i (inverse) exactly
template <class R>
__device__ __forceinline__ cx<R> cmul_negi(cx<R> a) { return {a.im, rneg(a.re)}; }
template <class R>
__device__ __forceinline__ cx<R> cmul_posi(cx<R> a) { return {rneg(a.im), a.re}; }
template <class R>
__device__ __forceinline__ cx<R> cconj(cx<R> a) { return {a.re, rneg(a.im)}; }
// a * w or a * conj(w)
template <class R>
__device__ __forceinline__ cx<R> cmul(cx<R> a, cx<R> w)
{
    return {rsub(rmul(a.re, w.re), rmul(a.im, w.im)), radd(rmul(a.re, w.im), rmul(a.im, w.re))};
}
template <class R>
__device__ __forceinline__ cx<R> cmulc(cx<R> a, cx<R> w)
{
    return {radd(rmul(a.re, w.re), rmul(a.im, w.im)), rsub(rmul(a.im, w.re), rmul(a.re, w.im))};
}
__device__ __forceinline__ cx<double> cmul(cx<double> a, cx<double> w)
{
    return {fma(a.re, w.re, -a.im * w.im), fma(a.re, w.im, a.im * w.re)};
}
__device__ __forceinline__ cx<double> cmulc(cx<double> a, cx<double> w)
{
    return {fma(a.re, w.re, a.im * w.im), fma(a.im, w.re, -a.re * w.im)};
}
__device__ __forceinline__ cx<float> cmul(cx<float> a, cx<float> w)
{
    return {fmaf(a.re, w.re, -a.im * w.im), fmaf(a.re, w.im, a.im * w.re)};
}
__device__ __forceinline__ cx<float> cmulc(cx<float> a, cx<float> w)
{
    return {fmaf(a.re, w.re, a.im * w.im), fmaf(a.im, w.re, -a.re * w.im)};
}
template <class R>
__device__ __forceinline__ cx<R> cscale(cx<R> a, R m) { return {rmul(a.re, m), rmul(a.im, m)}; }
template <class R>
__device__ __forceinline__ cx<R> cmulk(cx<R> a, double k) { return {rmulk(a.re, k), rmulk(a.im, k)}; }

// ------------------------------------------------------------------ policies
struct F64 {
    using real = double;
    using scplx = double2;
    using tw_t = double2;
    using mult_t = double;
    using io_t = double;
    static constexpr int kId = 0;
    static constexpr int kPadShift = 3;   // one pad element per 8 (128 bytes)
    // pruned first (zero-padded) and last (cropped) stages: they pay where the
    // arithmetic pipe is the limit, FP64 here
    static constexpr bool kPrune = true;       // x and y passes
    static constexpr bool kPruneConv = true;   // conv pass
    __device__ static __forceinline__ cx<real> ld(const scplx &v) { return {v.x, v.y}; }
    __device__ static __forceinline__ scplx st(cx<real> a) { return make_double2(a.re, a.im); }
    __device__ static __forceinline__ cx<real> tw(const tw_t &v) { return {v.x, v.y}; }
    __device__ static __forceinline__ real mult(mult_t m) { return m; }
    __device__ static __forceinline__ real from_io(io_t x) { return x; }
    __device__ static __forceinline__ io_t to_io(real x) { return x; }
    __device__ static __forceinline__ real zero() { return 0.0; }
};

struct F32 {
    using real = float;
    using scplx = float2;
    using tw_t = float2;
    using mult_t = float;
    using io_t = float;
    static constexpr int kId = 1;
    static constexpr int kPadShift = 4;   // one pad element per 16 (128 bytes)
    static constexpr bool kPrune = false;
    static constexpr bool kPruneConv = false;
    __device__ static __forceinline__ cx<real> ld(const scplx &v) { return {v.x, v.y}; }
    __device__ static __forceinline__ scplx st(cx<real> a) { return make_float2(a.re, a.im); }
    __device__ static __forceinline__ cx<real> tw(const tw_t &v) { return {v.x, v.y}; }
    __device__ static __forceinline__ real mult(mult_t m) { return m; }
    __device__ static __forceinline__ real from_io(io_t x) { return x; }
    __device__ static __forceinline__ io_t to_io(real x) { return x; }
    __device__ static __forceinline__ real zero() { return 0.0f; }
};

struct DF64 {
    using real = df;
    using scplx = float4;   // (re.hi, re.lo, im.hi, im.lo)
    using tw_t = float4;
    using mult_t = float2;  // (hi, lo)
    using io_t = double;
    static constexpr int kId = 2;
    static constexpr int kPadShift = 3;
    // pruning pays in the conv pass (measured 9 %); in the x and y passes,
    // which wait on memory more than on arithmetic, it made them slower
    static constexpr bool kPrune = false;
    static constexpr bool kPruneConv = true;
    __device__ static __forceinline__ cx<real> ld(const scplx &v) { return {df{v.x, v.y}, df{v.z, v.w}}; }
    // stored values are renormalised, so the unnormalised parts of the pair
    // arithmetic only live within one stage (fast_two_sum: see there)
    __device__ static __forceinline__ scplx st(cx<real> a)
    {
        float4 r;
        fast_two_sum(a.re.hi, a.re.lo, r.x, r.y);
        fast_two_sum(a.im.hi, a.im.lo, r.z, r.w);
        return r;
    }
    __device__ static __forceinline__ cx<real> tw(const tw_t &v) { return {df{v.x, v.y}, df{v.z, v.w}}; }
    __device__ static __forceinline__ real mult(mult_t m) { return df{m.x, m.y}; }
    __device__ static __forceinline__ real from_io(io_t x)
    {
        float h = __double2float_rn(x);
        float l = __double2float_rn(x - (double)h);
        return df{h, l};
    }
    __device__ static __forceinline__ io_t to_io(real x) { return df_to_double(x); }
    __device__ static __forceinline__ real zero() { return df{0.0f, 0.0f}; }
};

}  // namespace gsm
