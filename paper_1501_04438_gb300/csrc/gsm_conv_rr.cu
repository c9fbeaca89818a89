// gsm_conv_rr.cu -- the conv pass (Eq. I1FFT: forward FFT of the zero-padded
// line, multiplier, inverse FFT, crop) for FP32 lines of padded length 512,
// register-resident.
//
// The Stockham engine moves every element through shared memory once per
// radix stage; in FP32 that shared-memory traffic, not arithmetic, bounds the
// pass.  Here a line of 512 is held by 16 threads, 32 complex values each, and
// each transform goes through shared memory once:
//   forward, with z = t + 16 m (thread t, m = 0..31; x = 0 for m >= 16) and
//   k = k1 + 32 k2:
//     Y[k1 + 32 k2] = sum_t w16^(t k2) [ w512^(t k1) sum_m x[t + 16 m] w32^(m k1) ]
//     (thread t: DFT32 over m, twiddle w512^(t k1); transpose; thread t' takes
//     the rows k1 = t' and t' + 16: DFT16 over t);
//   multiplier in registers;
//   inverse, with n = a + 16 b:
//     z[a + 16 b] = sum_k1 w32^(-b k1) [ w512^(-a k1) sum_k2 Y[k1 + 32 k2] w16^(-a k2) ]
//     (inverse DFT16 over k2 per row, twiddle, transpose back, thread a: inverse
//     DFT32 over k1, only the outputs b < 16 are formed: the crop).
// The 32- and 16-point DFTs are two-level (4 x 8 and 4 x 4) on the butterflies
// of gsm_fft.cuh with compile-time twiddles.
#include "gsm_internal.h"

namespace gsm {

namespace {

// cos(2 pi j / 32), j = 0..8 (exact decimal expansions, rounded by the compiler)
__host__ __device__ constexpr float c32_base(int j)
{
    return j == 0   ? 1.0f
           : j == 1 ? 0.980785280403230449126182236134239037f
           : j == 2 ? 0.923879532511286756128183189396788933f
           : j == 3 ? 0.831469612302545237078788377617905756f
           : j == 4 ? 0.707106781186547524400844362104849039f
           : j == 5 ? 0.555570233019602224742830813948532875f
           : j == 6 ? 0.382683432365089771728459984030398867f
           : j == 7 ? 0.195090322016128267848284868477022241f
                    : 0.0f;
}

// cos and sin of 2 pi e / 32 for any integer e, by quadrant symmetry
__host__ __device__ constexpr float c32(int e)
{
    const int j = ((e % 32) + 32) % 32;
    return j <= 8 ? c32_base(j) : j <= 16 ? -c32_base(16 - j) : j <= 24 ? -c32_base(j - 16) : c32_base(32 - j);
}
__host__ __device__ constexpr float s32(int e) { return c32(e - 8); }

// a * w32^E, w32 = exp(-+ 2 pi i / 32) (forward / inverse)
template <int E, bool FWD>
__device__ __forceinline__ cx<float> rot32(cx<float> a)
{
    constexpr int e = ((E % 32) + 32) % 32;
    if constexpr (e == 0) {
        return a;
    } else if constexpr (e == 8) {          // -+ i
        return FWD ? cx<float>{a.im, -a.re} : cx<float>{-a.im, a.re};
    } else if constexpr (e == 16) {
        return {-a.re, -a.im};
    } else if constexpr (e == 24) {         // +- i
        return FWD ? cx<float>{-a.im, a.re} : cx<float>{a.im, -a.re};
    } else {
        constexpr float c = c32(e), s = s32(e);
        // forward: a (c - i s); inverse: a (c + i s)
        return FWD ? cx<float>{fmaf(a.re, c, a.im * s), fmaf(a.im, c, -a.re * s)}
                   : cx<float>{fmaf(a.re, c, -a.im * s), fmaf(a.im, c, a.re * s)};
    }
}

template <int M2, int K1, bool FWD>
__device__ __forceinline__ void tw32(cx<float> &a) { a = rot32<M2 * K1, FWD>(a); }

// 32-point DFT in registers, v[m] -> v[k] (natural order), as 4 x 8: inputs
// m = 8 m1 + m2, outputs k = k1 + 4 k2.  HALF_IN: v[16..31] are zero (not
// read); HALF_OUT: only the outputs k < 16 are formed.
template <bool FWD, bool HALF_IN, bool HALF_OUT>
__device__ __forceinline__ void dft32(cx<float> *v)
{
    cx<float> a[8][4];
#pragma unroll
    for (int m2 = 0; m2 < 8; ++m2) {
        a[m2][0] = v[m2];
        a[m2][1] = v[8 + m2];
        if (HALF_IN) {
            bfly<float, 4, FWD, 1>(a[m2]);
        } else {
            a[m2][2] = v[16 + m2];
            a[m2][3] = v[24 + m2];
            bfly<float, 4, FWD, 0>(a[m2]);
        }
    }
    // twiddles w32^(m2 k1)
#pragma unroll
    for (int m2 = 1; m2 < 8; ++m2) {
#pragma unroll
        for (int k1 = 1; k1 < 4; ++k1) {
            switch (m2 * k1) {   // resolved at compile time after unrolling
#define GSM_T(E) \
    case E: a[m2][k1] = rot32<E, FWD>(a[m2][k1]); break;
                GSM_T(1) GSM_T(2) GSM_T(3) GSM_T(4) GSM_T(5) GSM_T(6) GSM_T(7) GSM_T(8) GSM_T(9)
                GSM_T(10) GSM_T(12) GSM_T(14) GSM_T(15) GSM_T(18) GSM_T(21)
#undef GSM_T
            default: break;
            }
        }
    }
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
        cx<float> b[8];
#pragma unroll
        for (int m2 = 0; m2 < 8; ++m2) b[m2] = a[m2][k1];
        if (HALF_OUT) {
            bfly<float, 8, FWD, 2>(b);
#pragma unroll
            for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = b[k2];
        } else {
            bfly<float, 8, FWD, 0>(b);
#pragma unroll
            for (int k2 = 0; k2 < 8; ++k2) v[k1 + 4 * k2] = b[k2];
        }
    }
}

// 16-point DFT in registers, v[m] -> v[k] (natural order), as 4 x 4: inputs
// m = 4 m1 + m2, outputs k = k1 + 4 k2, twiddles w16^(m2 k1) = w32^(2 m2 k1).
template <bool FWD>
__device__ __forceinline__ void dft16(cx<float> *v)
{
    cx<float> a[4][4];
#pragma unroll
    for (int m2 = 0; m2 < 4; ++m2) {
#pragma unroll
        for (int m1 = 0; m1 < 4; ++m1) a[m2][m1] = v[4 * m1 + m2];
        bfly<float, 4, FWD, 0>(a[m2]);
    }
#pragma unroll
    for (int m2 = 1; m2 < 4; ++m2) {
#pragma unroll
        for (int k1 = 1; k1 < 4; ++k1) {
            switch (m2 * k1) {
#define GSM_T(E) \
    case E: a[m2][k1] = rot32<2 * E, FWD>(a[m2][k1]); break;
                GSM_T(1) GSM_T(2) GSM_T(3) GSM_T(4) GSM_T(6) GSM_T(9)
#undef GSM_T
            default: break;
            }
        }
    }
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
        cx<float> b[4] = {a[0][k1], a[1][k1], a[2][k1], a[3][k1]};
        bfly<float, 4, FWD, 0>(b);
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = b[k2];
    }
}

constexpr int kRrLinesPerCta = 16;           // 16 lines x 16 threads = 256 threads
constexpr int kRrRow = 17;                   // row pitch of the transpose buffer (bank spread)
constexpr int kRrLineElems = 32 * kRrRow;    // one line's transpose buffer

// One line of padded length 512 (n = 256 stored values) per 16 threads.
// Multiplier of frequency k: mrow[k] (full) or mrow[min(k, 512 - k)].
__global__ void __launch_bounds__(16 * kRrLinesPerCta, 2)
    k_conv_rr512(float2 *__restrict__ W, const float *__restrict__ mult, int nlines, int is3d, int My, int ny1,
                 int full, const float2 *__restrict__ tw)
{
    extern __shared__ float2 sbuf[];   // kRrLinesPerCta * kRrLineElems (dynamic: above 48 KB)
    const int t = threadIdx.x & 15;
    const int l = threadIdx.x >> 4;
    const int line = blockIdx.x * kRrLinesPerCta + l;
    const bool active = line < nlines;      // a whole half-warp, both take part in the syncs
    float2 *S = sbuf + l * kRrLineElems;
    float2 *w = W + (size_t)(active ? line : 0) * 256;
    const int ln = active ? line : 0;       // inactive lines read nothing past the tables
    const float *mrow;
    if (full) {
        mrow = mult + (size_t)ln * 512;
    } else if (is3d) {
        const int kx = ln / My, ky = ln - kx * My;
        mrow = mult + ((size_t)kx * ny1 + min(ky, My - ky)) * 257;
    } else {
        mrow = mult + (size_t)ln * 257;
    }

    // forward, step 1: DFT32 over m of x[t + 16 m] (m < 16 stored), twiddle w512^(t k1)
    cx<float> v[32];
#pragma unroll
    for (int m = 0; m < 16; ++m) {
        const float2 x = active ? w[t + 16 * m] : make_float2(0.f, 0.f);
        v[m] = {x.x, x.y};
    }
    dft32<true, true, false>(v);
#pragma unroll
    for (int k1 = 1; k1 < 32; ++k1) {
        const float2 q = tw[t * k1];
        v[k1] = cmul(v[k1], cx<float>{q.x, q.y});
    }
#pragma unroll
    for (int k1 = 0; k1 < 32; ++k1) S[k1 * kRrRow + t] = make_float2(v[k1].re, v[k1].im);
    __syncwarp();

    // forward, step 2: rows k1 = t and t + 16, DFT16 over the 16 threads' values;
    // multiplier; inverse step 2: DFT16 over k2, twiddle conj w512^(a k1)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int k1 = t + 16 * h;
        cx<float> *r = v + 16 * h;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const float2 x = S[k1 * kRrRow + i];
            r[i] = {x.x, x.y};
        }
        dft16<true>(r);
#pragma unroll
        for (int k2 = 0; k2 < 16; ++k2) {
            const int k = k1 + 32 * k2;
            const float m = active ? mrow[full ? k : min(k, 512 - k)] : 0.f;
            r[k2] = {r[k2].re * m, r[k2].im * m};
        }
        dft16<false>(r);
#pragma unroll
        for (int a = 1; a < 16; ++a) {
            const float2 q = tw[a * k1];
            r[a] = cmulc(r[a], cx<float>{q.x, q.y});
        }
    }
    __syncwarp();
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int k1 = t + 16 * h;
#pragma unroll
        for (int a = 0; a < 16; ++a) S[k1 * kRrRow + a] = make_float2(v[16 * h + a].re, v[16 * h + a].im);
    }
    __syncwarp();

    // inverse, step 1: thread a takes column a, inverse DFT32 over k1, outputs b < 16
#pragma unroll
    for (int k1 = 0; k1 < 32; ++k1) {
        const float2 x = S[k1 * kRrRow + t];
        v[k1] = {x.x, x.y};
    }
    dft32<false, false, true>(v);
    if (active) {
#pragma unroll
        for (int b = 0; b < 16; ++b) w[t + 16 * b] = make_float2(v[b].re, v[b].im);
    }
}

}  // namespace

// Conv pass of an FP32 plan whose conv lines have padded length 512 (n = 256).
gsm_status_t launch_conv_rr512_f32(void *W, const void *mult, int nlines, int is3d, int My, int ny1, bool full,
                                   const void *tw, cudaStream_t st)
{
    const int blocks = (nlines + kRrLinesPerCta - 1) / kRrLinesPerCta;
    const size_t smem = sizeof(float2) * kRrLinesPerCta * kRrLineElems;
    static bool raised[64] = {};   // per device; setting it twice is harmless
    int dev = 0;
    GSM_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64 || !raised[dev]) {
        GSM_CUDA_TRY(cudaFuncSetAttribute(k_conv_rr512, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        if (dev >= 0 && dev < 64) raised[dev] = true;
    }
    k_conv_rr512<<<blocks, 16 * kRrLinesPerCta, smem, st>>>(static_cast<float2 *>(W), static_cast<const float *>(mult),
                                                         nlines, is3d, My, ny1, full ? 1 : 0,
                                                         static_cast<const float2 *>(tw));
    GSM_CUDA_TRY(cudaGetLastError());
    return GSM_OK;
}

}  // namespace gsm
