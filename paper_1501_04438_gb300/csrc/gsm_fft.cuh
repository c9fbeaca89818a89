// gsm_fft.cuh -- batched line FFTs in shared memory (all three precisions).
//
// A CTA holds `nl` lines of length M in shared memory, line l at offset
// l * LS, element i at pidx(i) (one pad element every 2^kPadShift elements, so
// that the strided accesses of the early stages spread over the banks); the
// FFT of each line is done by its own group of threads (see Group).
// The transform is a Stockham autosort FFT (self-sorting, no bit reversal):
// for a stage of radix R after stages whose radices multiply to Ns,
// butterfly b (0 <= b < M/R) reads x[b + t M/R], t = 0..R-1, multiplies
// element t by w^(j t) with j = b mod Ns and w = exp(-+2 pi i / (Ns R)),
// applies the radix-R DFT in registers and writes the outputs to
// (b - j) R + j + t Ns.  Every thread first loads all its butterflies,
// the group synchronises, then every thread stores: stages run in place.
//
// Unnormalised: forward uses exp(-2 pi i jk/M), inverse exp(+2 pi i jk/M).
#pragma once

#include <type_traits>

#include "gsm_arith.cuh"

namespace gsm {

constexpr int kMaxStages = 12;

// Radix schedule of one FFT length: stage st has radix r[st] (8, 4, 2, 5 or 3,
// in any order whose product is M).
struct Sched {
    int M;
    int nst;
    unsigned char r[kMaxStages];
};

template <class Pol>
__host__ __device__ __forceinline__ int pidx(int i) { return i + (i >> Pol::kPadShift); }

template <class Pol>
__host__ __device__ __forceinline__ int line_stride(int M) { return M + (M >> Pol::kPadShift) + 1; }

// math constants (exact decimal expansions, rounded by the compiler)
constexpr double kSqrtHalf = 0.707106781186547524400844362104849039;
constexpr double kSin60 = 0.866025403784438646763723170752936183;  // sqrt(3)/2
constexpr double kC5a = 0.309016994374947424102293417182819059;    // cos(2 pi/5)
constexpr double kC5b = -0.809016994374947424102293417182819059;   // cos(4 pi/5)
constexpr double kS5a = 0.951056516295153572116439333379382143;    // sin(2 pi/5)
constexpr double kS5b = 0.587785252292473129168705954639072769;    // sin(4 pi/5)

// ---------------------------------------------------------------- butterflies
// y_k = sum_t x_t exp(-+ 2 pi i t k / R), in place in v[0..R-1].

template <class R, bool FWD>
__device__ __forceinline__ void bfly2(cx<R> *v)
{
    cx<R> a = v[0];
    v[0] = cadd(a, v[1]);
    v[1] = csub(a, v[1]);
}

template <class R, bool FWD>
__device__ __forceinline__ cx<R> rot_quarter(cx<R> a)   // multiply by -i (fwd) / +i (inv)
{
    return FWD ? cmul_negi(a) : cmul_posi(a);
}

template <class R, bool FWD>
__device__ __forceinline__ void bfly4(cx<R> *v)
{
    cx<R> a0 = cadd(v[0], v[2]), a1 = csub(v[0], v[2]);
    cx<R> a2 = cadd(v[1], v[3]), a3 = rot_quarter<R, FWD>(csub(v[1], v[3]));
    v[0] = cadd(a0, a2);
    v[2] = csub(a0, a2);
    v[1] = cadd(a1, a3);
    v[3] = csub(a1, a3);
}

// Radix 8, plain form: the rotations by w8 and w8^3 are formed first (used
// for FP32 and double-float, whose passes are not limited by arithmetic).
template <class R, bool FWD>
__device__ __forceinline__ void bfly8_plain(cx<R> *v)
{
    cx<R> a[4], b[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        a[t] = cadd(v[t], v[t + 4]);
        b[t] = csub(v[t], v[t + 4]);
    }
    {
        cx<R> z = b[1];
        if (FWD) b[1] = {rmulk(radd(z.re, z.im), kSqrtHalf), rmulk(rsub(z.im, z.re), kSqrtHalf)};
        else b[1] = {rmulk(rsub(z.re, z.im), kSqrtHalf), rmulk(radd(z.re, z.im), kSqrtHalf)};
    }
    b[2] = rot_quarter<R, FWD>(b[2]);
    {
        cx<R> z = b[3];
        if (FWD) b[3] = {rmulk(rsub(z.im, z.re), kSqrtHalf), rneg(rmulk(radd(z.re, z.im), kSqrtHalf))};
        else b[3] = {rneg(rmulk(radd(z.re, z.im), kSqrtHalf)), rmulk(rsub(z.re, z.im), kSqrtHalf)};
    }
    bfly4<R, FWD>(a);
    bfly4<R, FWD>(b);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        v[2 * k] = a[k];
        v[2 * k + 1] = b[k];
    }
}

// Radix 8 as two radix-4 transforms of a_t = x_t + x_{t+4} (even outputs)
// and of b_t = (x_t - x_{t+4}) w8^t (odd outputs).  The 1/sqrt(2) of w8 and
// w8^3 is applied in the last additions (x + c s contracts to one FMA; used
// for FP64, whose passes are limited by the FP64 pipe):
//   u1 = b1 w8 sqrt2, u3 = b3 w8^3 sqrt2 (additions only),
//   B0,2 = (b0 + b2') +- c (u1 + u3),  B1,3 = (b0 - b2') +- c rot(u1 - u3).
template <class R, bool FWD>
__device__ __forceinline__ void bfly8_odd(const cx<R> &b0, const cx<R> &b1, const cx<R> &b2, const cx<R> &b3,
                                          cx<R> *B, bool half)
{
    cx<R> u1, u3;
    if (FWD) {   // w8 = (1 - i)/sqrt2, w8^3 = (-1 - i)/sqrt2
        u1 = {radd(b1.re, b1.im), rsub(b1.im, b1.re)};
        u3 = {rsub(b3.im, b3.re), rneg(radd(b3.re, b3.im))};
    } else {     // conjugates
        u1 = {rsub(b1.re, b1.im), radd(b1.re, b1.im)};
        u3 = {rneg(radd(b3.re, b3.im)), rsub(b3.re, b3.im)};
    }
    const cx<R> b2r = rot_quarter<R, FWD>(b2);
    const cx<R> p = cadd(b0, b2r), q = csub(b0, b2r);
    const cx<R> s = cadd(u1, u3), d = rot_quarter<R, FWD>(csub(u1, u3));
    B[0] = {radd(p.re, rmulk(s.re, kSqrtHalf)), radd(p.im, rmulk(s.im, kSqrtHalf))};
    B[1] = {radd(q.re, rmulk(d.re, kSqrtHalf)), radd(q.im, rmulk(d.im, kSqrtHalf))};
    if (half) return;
    B[2] = {rsub(p.re, rmulk(s.re, kSqrtHalf)), rsub(p.im, rmulk(s.im, kSqrtHalf))};
    B[3] = {rsub(q.re, rmulk(d.re, kSqrtHalf)), rsub(q.im, rmulk(d.im, kSqrtHalf))};
}

template <class R, bool FWD>
__device__ __forceinline__ void bfly8(cx<R> *v)
{
    cx<R> a[4], b[4], B[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        a[t] = cadd(v[t], v[t + 4]);
        b[t] = csub(v[t], v[t + 4]);
    }
    bfly4<R, FWD>(a);
    bfly8_odd<R, FWD>(b[0], b[1], b[2], b[3], B, false);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        v[2 * k] = a[k];
        v[2 * k + 1] = B[k];
    }
}

// --- pruned butterflies -------------------------------------------------------
// First stage of a transform whose inputs x_t, t >= R/2, are zero (zero
// padding): a_t = b_t = x_t.  Last stage of a transform of which only the
// outputs t < R/2 are kept (the crop): the other outputs are not formed.
template <class R, bool FWD>
__device__ __forceinline__ void bfly8_half_in(cx<R> *v)
{
    cx<R> a[4] = {v[0], v[1], v[2], v[3]}, B[4];
    bfly4<R, FWD>(a);
    bfly8_odd<R, FWD>(v[0], v[1], v[2], v[3], B, false);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        v[2 * k] = a[k];
        v[2 * k + 1] = B[k];
    }
}

template <class R, bool FWD>
__device__ __forceinline__ void bfly8_half_out(cx<R> *v)
{
    cx<R> a[4], b[4], B[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        a[t] = cadd(v[t], v[t + 4]);
        b[t] = csub(v[t], v[t + 4]);
    }
    // outputs 0 and 1 of the radix-4 transform of a
    const cx<R> p = cadd(a[0], a[2]), q = csub(a[0], a[2]);
    const cx<R> s = cadd(a[1], a[3]), d = rot_quarter<R, FWD>(csub(a[1], a[3]));
    bfly8_odd<R, FWD>(b[0], b[1], b[2], b[3], B, true);
    v[0] = cadd(p, s);
    v[1] = B[0];
    v[2] = cadd(q, d);
    v[3] = B[1];
}

template <class R, bool FWD>
__device__ __forceinline__ void bfly4_half_in(cx<R> *v)
{
    const cx<R> x0 = v[0], x1 = v[1], r1 = rot_quarter<R, FWD>(v[1]);
    v[0] = cadd(x0, x1);
    v[1] = cadd(x0, r1);
    v[2] = csub(x0, x1);
    v[3] = csub(x0, r1);
}

template <class R, bool FWD>
__device__ __forceinline__ void bfly4_half_out(cx<R> *v)
{
    const cx<R> p = cadd(v[0], v[2]), q = csub(v[0], v[2]);
    const cx<R> s = cadd(v[1], v[3]), d = rot_quarter<R, FWD>(csub(v[1], v[3]));
    v[0] = cadd(p, s);
    v[1] = cadd(q, d);
}

template <class R, bool FWD>
__device__ __forceinline__ void bfly2_half_in(cx<R> *v) { v[1] = v[0]; }

template <class R, bool FWD>
__device__ __forceinline__ void bfly2_half_out(cx<R> *v) { v[0] = cadd(v[0], v[1]); }

template <class R, bool FWD>
__device__ __forceinline__ void bfly3(cx<R> *v)
{
    cx<R> s = cadd(v[1], v[2]);
    cx<R> d = csub(v[1], v[2]);
    cx<R> y0 = cadd(v[0], s);
    cx<R> m = csub(v[0], cmulk(s, 0.5));
    cx<R> r = rot_quarter<R, FWD>(cmulk(d, kSin60));   // -+ i (sqrt3/2)(x1 - x2)
    v[0] = y0;
    v[1] = cadd(m, r);
    v[2] = csub(m, r);
}

template <class R, bool FWD>
__device__ __forceinline__ void bfly5(cx<R> *v)
{
    cx<R> a1 = cadd(v[1], v[4]), b1 = csub(v[1], v[4]);
    cx<R> a2 = cadd(v[2], v[3]), b2 = csub(v[2], v[3]);
    cx<R> x0 = v[0];
    cx<R> p1 = cadd(x0, cadd(cmulk(a1, kC5a), cmulk(a2, kC5b)));
    cx<R> p2 = cadd(x0, cadd(cmulk(a1, kC5b), cmulk(a2, kC5a)));
    cx<R> q1 = rot_quarter<R, FWD>(cadd(cmulk(b1, kS5a), cmulk(b2, kS5b)));   // -+ i (s1 b1 + s2 b2)
    cx<R> q2 = rot_quarter<R, FWD>(csub(cmulk(b1, kS5b), cmulk(b2, kS5a)));   // -+ i (s2 b1 - s1 b2)
    v[0] = cadd(x0, cadd(a1, a2));
    v[1] = cadd(p1, q1);
    v[4] = csub(p1, q1);
    v[2] = cadd(p2, q2);
    v[3] = csub(p2, q2);
}

// HALF = 0: full radix-RAD DFT; 1: inputs t >= RAD/2 are zero; 2: only the
// outputs t < RAD/2 are formed (even RAD only).
template <class R, int RAD, bool FWD, int HALF>
__device__ __forceinline__ void bfly(cx<R> *v)
{
    if constexpr (RAD == 2) {
        if constexpr (HALF == 1) bfly2_half_in<R, FWD>(v);
        else if constexpr (HALF == 2) bfly2_half_out<R, FWD>(v);
        else bfly2<R, FWD>(v);
    } else if constexpr (RAD == 3) {
        bfly3<R, FWD>(v);
    } else if constexpr (RAD == 4) {
        if constexpr (HALF == 1) bfly4_half_in<R, FWD>(v);
        else if constexpr (HALF == 2) bfly4_half_out<R, FWD>(v);
        else bfly4<R, FWD>(v);
    } else if constexpr (RAD == 5) {
        bfly5<R, FWD>(v);
    } else {
        if constexpr (HALF == 1) bfly8_half_in<R, FWD>(v);
        else if constexpr (HALF == 2) bfly8_half_out<R, FWD>(v);
        else if constexpr (std::is_same<R, double>::value) bfly8<R, FWD>(v);
        else bfly8_plain<R, FWD>(v);
    }
}

// ---------------------------------------------------------------- groups
// The FFT of one line is done by a group of T threads (a multiple of 32).
// The group synchronises with __syncwarp (one warp), with __syncthreads
// (the group is the whole CTA) or with a named barrier of its own, so groups
// of one CTA never wait for each other between stages.
struct Group {
    int t;      // thread index in the group
    int T;      // threads in the group
    int bar;    // -1: one warp; 0: whole CTA; > 0: named barrier id
};

__device__ __forceinline__ void group_sync(const Group &g)
{
    if (g.bar < 0) __syncwarp();
    else if (g.bar == 0) __syncthreads();
    else asm volatile("bar.sync %0, %1;" ::"r"(g.bar), "r"(g.T) : "memory");
}

// Group of the calling thread when the CTA holds nl groups of T threads each.
__device__ __forceinline__ Group make_group(int T, int nl)
{
    Group g;
    g.t = threadIdx.x % T;
    g.T = T;
    g.bar = (T == 32) ? -1 : (nl == 1 ? 0 : 1 + (int)(threadIdx.x / T));
    return g;
}

// b mod Ns; the radix-8/4/2 stages come first, so Ns is usually a power of two
__device__ __forceinline__ int stage_mod(int b, int Ns)
{
    return (Ns & (Ns - 1)) == 0 ? (b & (Ns - 1)) : b % Ns;
}

// ---------------------------------------------------------------- one stage
// One Stockham stage on one line s[pidx(0..M-1)] by the group.  NB = upper
// bound of butterflies per thread (compile time); every thread first loads
// its butterflies, the group synchronises, then every thread stores.
// HALF = 1 (first stage of a zero-padded transform): only the inputs t < RAD/2
// are read; HALF = 2 (last stage of a cropped transform): only the outputs
// t < RAD/2, which land in the first half of the line, are formed and stored.
template <class Pol, int RAD, bool FWD, int NB, int HALF>
__device__ __forceinline__ void fft_stage(typename Pol::scplx *s, int M, int Ns,
                                          const typename Pol::tw_t *__restrict__ tw, const Group &g)
{
    using R = typename Pol::real;
    constexpr int NIN = HALF == 1 ? RAD / 2 : RAD;
    constexpr int NOUT = HALF == 2 ? RAD / 2 : RAD;
    const int nb = M / RAD;
    const int step = M / (Ns * RAD);   // twiddle-table stride of this stage
    cx<R> v[NB][RAD];
#pragma unroll
    for (int i = 0; i < NB; ++i) {
        const int b = g.t + i * g.T;
        if (b < nb) {
#pragma unroll
            for (int t = 0; t < NIN; ++t) v[i][t] = Pol::ld(s[pidx<Pol>(b + t * nb)]);
            if (Ns > 1) {
                const int j = stage_mod(b, Ns);
#pragma unroll
                for (int t = 1; t < NIN; ++t) {
                    cx<R> w = Pol::tw(tw[j * t * step]);
                    v[i][t] = FWD ? cmul(v[i][t], w) : cmulc(v[i][t], w);
                }
            }
            bfly<R, RAD, FWD, HALF>(v[i]);
        }
    }
    group_sync(g);
#pragma unroll
    for (int i = 0; i < NB; ++i) {
        const int b = g.t + i * g.T;
        if (b < nb) {
            const int j = stage_mod(b, Ns);
            const int d0 = (b - j) * RAD + j;
#pragma unroll
            for (int t = 0; t < NOUT; ++t) s[pidx<Pol>(d0 + t * Ns)] = Pol::st(v[i][t]);
        }
    }
    group_sync(g);
}

// ---------------------------------------------------------------- FMA-form stages (FP64)
// FMA-form constants exist for the twiddled stages (Ns > 1) of radix 8 and 4,
// and of radix 2 when Ns is even, that is whenever D = R Ns is a multiple of 4,
// so that the nearest quarter turn of every twiddle is exact: gslots(R) slots
// for each index j < Ns, rounded up to whole blocks of kGBlk indices, stage
// after stage in schedule order.
__host__ __device__ __forceinline__ bool gtabled(int R) { return R == 8 || R == 4 || R == 2; }
__host__ __device__ __forceinline__ bool gtabled_at(int R, long Ns)
{
    return Ns > 1 && gtabled(R) && ((long)R * Ns) % 4 == 0;
}
__host__ __device__ __forceinline__ int gslots(int R) { return R == 8 ? 16 : (R == 4 ? 8 : 4); }
constexpr int kGBlk = 32;

// Doubles of the constants of one stage of radix R after stages of product Ns.
__host__ __device__ __forceinline__ size_t gblock(int R, size_t Ns)
{
    return (Ns + kGBlk - 1) / kGBlk * kGBlk * (size_t)gslots(R);
}

// First slot of index j within a stage's constants.
__host__ __device__ __forceinline__ size_t gindex(int R, size_t j)
{
    return (j / kGBlk) * (size_t)(gslots(R) * kGBlk) + j % kGBlk;
}

// Offset (in doubles) of the constants of stage st.
__host__ __device__ inline size_t gtable_offset(const Sched &sc, int st)
{
    size_t off = 0, Ns = 1;
    for (int i = 0; i < st && i < sc.nst; ++i) {
        if (gtabled_at(sc.r[i], (long)Ns)) off += gblock(sc.r[i], Ns);
        Ns *= (size_t)sc.r[i];
    }
    return off;
}

// Doubles of all FMA-form constants of a schedule.
inline size_t g8_table_doubles(const Sched &sc) { return gtable_offset(sc, sc.nst); }

// Twiddled stages in which every multiplication is fused into an addition:
// the "tangent" form of the twiddle factors (E. N. Linzer and E. Feig, IEEE
// Trans. Signal Process. 41 (1993); S. Goedecker, SIAM J. Sci. Comput. 18
// (1997)).  Each twiddle W_t = w^(jt) is written
//   W_t = f_t i^(k_t) (1 + i tau_t),  |tau_t| <= 1,  f_t = cos(phi_t) >= 1/sqrt2,
// with i^(k_t) the nearest quarter turn.  X_t = i^(k_t)(1 + i tau_t) x_t costs
// two FMAs (the quarter turn is a swap and sign flips, done on the integer
// side); the real scales f_t are carried as ratios through the butterfly's
// layers, each a pair of FMAs per complex value, and cancel at the end because
// f_0 = 1.  Radix 8: 66 FP64 instructions per butterfly instead of 80;
// radix 4: 22 instead of 28; radix 2: 6 instead of 8.  A stage's constants
// are slot-major in blocks of kGBlk = 32 indices: slot q of index j is at
// ((j / 32) * slots + q) * 32 + j % 32, so the threads of a warp, which hold
// consecutive j, read each slot from 256 consecutive bytes (two 128-byte
// lines per warp instead of one line per thread), and a thread reaches its
// slots at fixed offsets from one pointer.  Slots
// (forward direction; the inverse uses conj(W_t) = f_t i^(-k_t)(1 - i tau_t)):
//   radix 8 (16 slots): 0..6 tau_t sigma_t (t = 1..7;
//     sigma_t = -1 for odd k_t, which folds the swap's sign into the tangent),
//     7..10 r_t = f_(t+4) / f_t (t = 0..3), 11 f_2, 12 f_3 / f_1, 13 f_1,
//     14 f_1 / sqrt2, 15 the codes k_t mod 4 in bits 2(t-1), 2(t-1)+1 (an
//     integer in the double's bits);
//   radix 4 (8 slots): tau_t sigma_t (t = 1..3), f_2, f_3 / f_1, f_1, codes, -;
//   radix 2 (4 slots): tau_1 sigma_1, f_1, code, -.
// Slot q of the constants at c (index j's first slot).
__device__ __forceinline__ double gslot(const double *__restrict__ c, int q) { return __ldg(c + q * kGBlk); }

__device__ __forceinline__ double flip_sign(double x, unsigned neg)
{
    return __hiloint2double(__double2hiint(x) ^ (int)(neg << 31), __double2loint(x));
}

// i^k (1 + i tt) x with tt the signed tangent of the stored convention.
__device__ __forceinline__ cx<double> tangent_rot(cx<double> x, int k, double tt)
{
    const bool sw = k & 1;
    const double a = sw ? x.im : x.re, b = sw ? x.re : x.im;
    const double re = fma(-tt, b, a), im = fma(tt, a, b);
    return {flip_sign(re, (unsigned)((k ^ (k >> 1)) & 1)), flip_sign(im, (unsigned)((k >> 1) & 1))};
}

// In-place DFT4 of z_0..z_3 carried as z_t = h_t zh_t with h_0 = 1 (ratios
// q2 = h_2, q31 = h_3 / h_1, q1 = h_1): z_n <- Z_n; with HALFOUT only Z_0, Z_1.
template <bool FWD, bool HALFOUT>
__device__ __forceinline__ void dft4_scaled(cx<double> &z0, cx<double> &z1, cx<double> &z2, cx<double> &z3,
                                            double q2, double q31, double q1)
{
    const cx<double> P = {fma(q2, z2.re, z0.re), fma(q2, z2.im, z0.im)};
    const cx<double> Q = {fma(-q2, z2.re, z0.re), fma(-q2, z2.im, z0.im)};
    const cx<double> R = {fma(q31, z3.re, z1.re), fma(q31, z3.im, z1.im)};
    const cx<double> S = {fma(-q31, z3.re, z1.re), fma(-q31, z3.im, z1.im)};
    // Z_1 = Q -+ i S (forward: -i), Z_3 = Q +- i S
    const cx<double> iS = FWD ? cx<double>{S.im, -S.re} : cx<double>{-S.im, S.re};
    z0 = {fma(q1, R.re, P.re), fma(q1, R.im, P.im)};
    z1 = {fma(q1, iS.re, Q.re), fma(q1, iS.im, Q.im)};
    if (!HALFOUT) {
        z2 = {fma(-q1, R.re, P.re), fma(-q1, R.im, P.im)};
        z3 = {fma(-q1, iS.re, Q.re), fma(-q1, iS.im, Q.im)};
    }
}

// One twiddled radix-8 butterfly in FMA form, in place: v[0..7] in,
// Y_0..Y_(NOUT-1) out.  Constants are read where they are used.
template <bool FWD, int NOUT>
__device__ __forceinline__ void bfly8_fma(cx<double> *v, const double *__restrict__ c)
{
    const int codes = __double2loint(gslot(c, 15));
#pragma unroll
    for (int t = 1; t < 8; ++t) {
        int k = (codes >> (2 * (t - 1))) & 3;
        if (!FWD) k = (4 - k) & 3;
        const double tt = gslot(c, t - 1);
        v[t] = tangent_rot(v[t], k, FWD ? tt : -tt);
    }
    // layer 1: v_t <- E_t = X_t + r_t X_(t+4) (scale f_t), v_(t+4) <- O_t = X_t - r_t X_(t+4)
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        const double r = gslot(c, 7 + t);
        const cx<double> x = v[t], y = v[t + 4];
        v[t] = {fma(r, y.re, x.re), fma(r, y.im, x.im)};
        v[t + 4] = {fma(-r, y.re, x.re), fma(-r, y.im, x.im)};
    }
    // odd branch: O_t w8^t; the 1/sqrt2 of w8, w8^3 joins the scale of O_1, O_3
    {
        const cx<double> a = v[5], d = v[6], b = v[7];
        if (FWD) {
            v[5] = {a.re + a.im, a.im - a.re};        // (1 - i) a
            v[6] = {d.im, -d.re};                     // -i d
            v[7] = {b.im - b.re, -b.im - b.re};       // (-1 - i) b
        } else {
            v[5] = {a.re - a.im, a.im + a.re};        // (1 + i) a
            v[6] = {-d.im, d.re};                     // i d
            v[7] = {-b.re - b.im, b.re - b.im};       // (-1 + i) b
        }
    }
    const double f2 = gslot(c, 11), f31 = gslot(c, 12);
    dft4_scaled<FWD, NOUT == 4>(v[0], v[1], v[2], v[3], f2, f31, gslot(c, 13));   // Y_0, Y_2, Y_4, Y_6
    dft4_scaled<FWD, NOUT == 4>(v[4], v[5], v[6], v[7], f2, f31, gslot(c, 14));   // Y_1, Y_3, Y_5, Y_7
    // interleave (register renaming only)
    const cx<double> e1 = v[1], e2 = v[2], e3 = v[3], o0 = v[4], o1 = v[5], o2 = v[6];
    v[1] = o0;
    v[2] = e1;
    v[3] = o1;
    if (NOUT == 8) {
        v[4] = e2;
        v[5] = o2;
        v[6] = e3;
    }
}

// Twiddled radix-4 butterfly in FMA form, in place (Y_0..Y_3 in natural
// order; HALFOUT: Y_0, Y_1 only).  Constant slots at c: tau_t sigma_t (t = 1..3),
// f_2, f_3 / f_1, f_1, the quarter-turn codes, one unused slot.
template <bool FWD, bool HALFOUT>
__device__ __forceinline__ void bfly4_fma(cx<double> *v, const double *__restrict__ c)
{
    const int codes = __double2loint(gslot(c, 6));
#pragma unroll
    for (int t = 1; t < 4; ++t) {
        int k = (codes >> (2 * (t - 1))) & 3;
        if (!FWD) k = (4 - k) & 3;
        const double tt = gslot(c, t - 1);
        v[t] = tangent_rot(v[t], k, FWD ? tt : -tt);
    }
    dft4_scaled<FWD, HALFOUT>(v[0], v[1], v[2], v[3], gslot(c, 3), gslot(c, 4), gslot(c, 5));
}

// Twiddled radix-2 butterfly in FMA form: Y_0,1 = x_0 +- f_1 X_1.  Constant
// slots at c: tau_1 sigma_1, f_1, the quarter-turn code, one unused slot.
template <bool FWD, bool HALFOUT>
__device__ __forceinline__ void bfly2_fma(cx<double> *v, const double *__restrict__ c)
{
    int k = __double2loint(gslot(c, 2)) & 3;
    if (!FWD) k = (4 - k) & 3;
    const double tt = gslot(c, 0);
    const cx<double> X = tangent_rot(v[1], k, FWD ? tt : -tt);
    const double f = gslot(c, 1);
    const cx<double> x0 = v[0];
    v[0] = {fma(f, X.re, x0.re), fma(f, X.im, x0.im)};
    if (!HALFOUT) v[1] = {fma(-f, X.re, x0.re), fma(-f, X.im, x0.im)};
}

// Twiddled Stockham stage of radix RAD (8, 4 or 2; gtabled_at(RAD, Ns)) in
// FMA form; HALF = 2: only the outputs t < RAD/2 (the crop).  Same data
// movement as fft_stage; gt points at this stage's constants.
template <int RAD, bool FWD, int NB, int HALF>
__device__ __forceinline__ void fft_stage_fma(double2 *s, int M, int Ns, const double *__restrict__ gt,
                                              const Group &g)
{
    constexpr int NOUT = HALF == 2 ? RAD / 2 : RAD;
    const int nb = M / RAD;
    cx<double> v[NB][RAD];
#pragma unroll
    for (int i = 0; i < NB; ++i) {
        const int b = g.t + i * g.T;
        if (b < nb) {
#pragma unroll
            for (int t = 0; t < RAD; ++t) v[i][t] = F64::ld(s[pidx<F64>(b + t * nb)]);
            const double *c = gt + gindex(RAD, stage_mod(b, Ns));
            if constexpr (RAD == 8) bfly8_fma<FWD, NOUT>(v[i], c);
            else if constexpr (RAD == 4) bfly4_fma<FWD, HALF == 2>(v[i], c);
            else bfly2_fma<FWD, HALF == 2>(v[i], c);
        }
    }
    group_sync(g);
#pragma unroll
    for (int i = 0; i < NB; ++i) {
        const int b = g.t + i * g.T;
        if (b < nb) {
            const int j = stage_mod(b, Ns);
            const int d0 = (b - j) * RAD + j;
#pragma unroll
            for (int t = 0; t < NOUT; ++t) s[pidx<F64>(d0 + t * Ns)] = F64::st(v[i][t]);
        }
    }
    group_sync(g);
}

// Rank of a radix in the order the stages of a schedule run in: 8, 4, 2, 5, 3.
__host__ __device__ __forceinline__ int radix_rank(int R)
{
    return R == 8 ? 0 : R == 4 ? 1 : R == 2 ? 2 : R == 5 ? 3 : R == 3 ? 4 : 99;
}

// Whether stages [from, nst) of sc are in the order 8, 4, 2, 5, 3 (radices of
// equal rank together), the only order fft_line runs.
__host__ __device__ inline bool sched_sorted_from(const Sched &sc, int from)
{
    for (int i = from; i < sc.nst; ++i) {
        if (radix_rank(sc.r[i]) > 4) return false;
        if (i > from && radix_rank(sc.r[i]) < radix_rank(sc.r[i - 1])) return false;
    }
    return true;
}

// All stages of the FFT of one line by one group.  EMAX bounds the elements
// per thread (M <= EMAX * T).  The caller synchronises the group (or CTA)
// after writing the line; the last stage ends with a group barrier, so the
// group may read the result right away.  The stages from st_begin on must be
// in the order 8, 4, 2, 5, 3 (sched_sorted_from, checked on the host): each
// radix gets one loop of its own, once (a loop mixing several large stage
// bodies, or one loop around these loops, costs the register allocator
// dearly: measured 11 % on the double-float passes).  Schedules that start
// with another radix (the inverse of a conv pass whose first stage is fused,
// fft_fused_mid) run from st_begin = 1.
// ZPAD: the second half of the input is zero and is not read (the first stage
// is pruned, so the first radix must be even); the caller need not write it.
// CROP: only the first half of the output is needed (the last stage is pruned
// when its radix is even; the second half of the line is then left
// undefined).  The caller chooses them per pass from the policy's kPrune
// (x and y passes) and kPruneConv (conv pass); without them the full stages
// run and the caller writes the zeros.
// gt (FP64 only, may be NULL): the constants of the FMA-form stages
// (fft_stage_fma), laid out as gtable_offset describes; with NULL every stage
// takes the twiddle table tw.  Stages [st_begin, st_end) run (st_end < 0: to
// the last).
template <class Pol, bool FWD, int EMAX, bool ZPAD_ = false, bool CROP_ = false>
__device__ __forceinline__ void fft_line(typename Pol::scplx *s, const Sched &sc,
                                         const typename Pol::tw_t *__restrict__ tw, const Group &g,
                                         const double *__restrict__ gt = nullptr, int st_begin = 0,
                                         int st_end = -1)
{
    constexpr bool ZPAD = ZPAD_, CROP = CROP_;
    const int M = sc.M, last = sc.nst - 1;
    const int nend = st_end < 0 ? sc.nst : st_end;   // stages [st_begin, nend) run
    int Ns = 1, st = st_begin;
    for (int i = 0; i < st_begin; ++i) Ns *= sc.r[i];
#define GSM_STAGE(RAD)                                                                         \
    do {                                                                                       \
        constexpr int NB = (EMAX + RAD - 1) / RAD;                                             \
        if (ZPAD && st == 0 && (RAD % 2) == 0)                                                 \
            fft_stage<Pol, RAD, FWD, NB, (RAD % 2 == 0) ? 1 : 0>(s, M, Ns, tw, g);             \
        else if (CROP && st == last && st > 0 && (RAD % 2) == 0)                               \
            fft_stage<Pol, RAD, FWD, NB, (RAD % 2 == 0) ? 2 : 0>(s, M, Ns, tw, g);             \
        else                                                                                   \
            fft_stage<Pol, RAD, FWD, NB, 0>(s, M, Ns, tw, g);                                  \
    } while (0)
    if constexpr (std::is_same<Pol, F64>::value) {
        if (gt != nullptr) {
            // the untwiddled first stage is peeled off so that each loop below
            // holds one FMA-form stage body
            if (st == 0 && st < nend) {
                const int r0 = sc.r[0];
                if (r0 == 8) GSM_STAGE(8);
                else if (r0 == 4) GSM_STAGE(4);
                else if (r0 == 2) GSM_STAGE(2);
                else if (r0 == 5) GSM_STAGE(5);
                else GSM_STAGE(3);
                st = 1;
                Ns = r0;
            }
            size_t goff = gtable_offset(sc, st);
            for (; st < nend && sc.r[st] == 8; ++st, Ns *= 8) {
                if (CROP && st == last) fft_stage_fma<8, FWD, (EMAX + 7) / 8, 2>(s, M, Ns, gt + goff, g);
                else fft_stage_fma<8, FWD, (EMAX + 7) / 8, 0>(s, M, Ns, gt + goff, g);
                goff += gblock(8, Ns);
            }
            for (; st < nend && sc.r[st] == 4; ++st, Ns *= 4) {
                if (CROP && st == last) fft_stage_fma<4, FWD, (EMAX + 3) / 4, 2>(s, M, Ns, gt + goff, g);
                else fft_stage_fma<4, FWD, (EMAX + 3) / 4, 0>(s, M, Ns, gt + goff, g);
                goff += gblock(4, Ns);
            }
            for (; st < nend && sc.r[st] == 2 && gtabled_at(2, Ns); ++st, Ns *= 2) {
                if (CROP && st == last) fft_stage_fma<2, FWD, (EMAX + 1) / 2, 2>(s, M, Ns, gt + goff, g);
                else fft_stage_fma<2, FWD, (EMAX + 1) / 2, 0>(s, M, Ns, gt + goff, g);
                goff += gblock(2, Ns);
            }
        }
    }
    for (; st < nend && sc.r[st] == 8; ++st, Ns *= 8) GSM_STAGE(8);
    for (; st < nend && sc.r[st] == 4; ++st, Ns *= 4) GSM_STAGE(4);
    for (; st < nend && sc.r[st] == 2; ++st, Ns *= 2) GSM_STAGE(2);
    for (; st < nend && sc.r[st] == 5; ++st, Ns *= 5) GSM_STAGE(5);
    for (; st < nend && sc.r[st] == 3; ++st, Ns *= 3) GSM_STAGE(3);
#undef GSM_STAGE
}

// The radix of the stage that fft_fused_mid can fuse for a transform whose
// forward schedule is scf and inverse schedule sci: the forward's last radix
// when the inverse starts with the same radix and both have at least two
// stages; 0 when they cannot be fused.
__host__ __device__ __forceinline__ int fused_radix(const Sched &scf, const Sched &sci)
{
    if (scf.nst < 2 || sci.nst < 2) return 0;
    const int R = scf.r[scf.nst - 1];
    return R == sci.r[0] ? R : 0;
}

// The last forward stage (radix R, schedule scf), a pointwise multiplication
// by mult(k) and the first inverse stage (radix R, schedule sci) of a line, in
// registers.  The forward stage's butterfly b (Ns = M/R = nb, so j = b and the
// twiddles are w_M^(b t)) leaves its outputs at the natural indices b + t M/R,
// which are exactly the inputs of the inverse's untwiddled butterfly b; that
// one writes to R b + t.  Saves two shared-memory round trips and a barrier
// over running the two transforms and the multiplication apart.  Follow with
// fft_line<Pol, false, ...>(..., sci, ..., st_begin = 1).
template <class Pol, int R, int NB, class MultF>
__device__ __forceinline__ void fft_fused_mid(typename Pol::scplx *s, const Sched &scf,
                                              const typename Pol::tw_t *__restrict__ tw, const Group &g,
                                              const double *__restrict__ gt, MultF mult)
{
    using Rl = typename Pol::real;
    const int M = scf.M, nb = M / R;
    cx<Rl> v[NB][R];
#pragma unroll
    for (int i = 0; i < NB; ++i) {
        const int b = g.t + i * g.T;
        if (b < nb) {
#pragma unroll
            for (int t = 0; t < R; ++t) v[i][t] = Pol::ld(s[pidx<Pol>(b + t * nb)]);
            bool done = false;
            if constexpr (std::is_same<Pol, F64>::value && (R == 8 || R == 4 || R == 2)) {
                if (gt != nullptr && gtabled_at(R, nb)) {
                    const double *c = gt + gtable_offset(scf, scf.nst - 1) + gindex(R, b);
                    if constexpr (R == 8) bfly8_fma<true, 8>(v[i], c);
                    else if constexpr (R == 4) bfly4_fma<true, false>(v[i], c);
                    else bfly2_fma<true, false>(v[i], c);
                    done = true;
                }
            }
            if (!done) {
#pragma unroll
                for (int t = 1; t < R; ++t) v[i][t] = cmul(v[i][t], Pol::tw(tw[b * t]));   // twiddle step 1
                bfly<Rl, R, true, 0>(v[i]);
            }
#pragma unroll
            for (int t = 0; t < R; ++t) v[i][t] = cscale(v[i][t], mult(b + t * nb));
            bfly<Rl, R, false, 0>(v[i]);
        }
    }
    group_sync(g);
#pragma unroll
    for (int i = 0; i < NB; ++i) {
        const int b = g.t + i * g.T;
        if (b < nb) {
#pragma unroll
            for (int t = 0; t < R; ++t) s[pidx<Pol>(R * b + t)] = Pol::st(v[i][t]);
        }
    }
    group_sync(g);
}

}  // namespace gsm
