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
#include <algorithm>

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
constexpr size_t kRrSmem = sizeof(float2) * kRrLinesPerCta * kRrLineElems;

// The 512-point transforms of one line by its 16 threads, in pieces (S is the
// line's transpose buffer; each thread reads and writes only its own rows
// k1 = t and t + 16, so row work needs no barrier):
//   fwd512_cols: on entry v[m] = x[t + 16 m], m < 16 (the rest is zero
//     padding); DFT32 over m, twiddle w512^(t k1), to S (column t), barrier.
//   fwd512_row: r[k2] = Y[k1 + 32 k2] for row k1 (a 16-point DFT of the row).
//   inv512_row: r holds Y[k1 + 32 k2]; inverse DFT16, twiddle, to S (row k1).
//   inv512_cols: barrier, column t from S, inverse DFT32 keeping the outputs
//     b < 16: v[b] = z[t + 16 b].
__device__ __forceinline__ void fwd512_cols(cx<float> *v, float2 *S, int t, const float2 *__restrict__ tw)
{
    dft32<true, true, false>(v);
#pragma unroll
    for (int k1 = 1; k1 < 32; ++k1) {
        const float2 q = tw[t * k1];
        v[k1] = cmul(v[k1], cx<float>{q.x, q.y});
    }
#pragma unroll
    for (int k1 = 0; k1 < 32; ++k1) S[k1 * kRrRow + t] = make_float2(v[k1].re, v[k1].im);
    __syncwarp();
}

__device__ __forceinline__ void fwd512_row(cx<float> *r, const float2 *S, int k1)
{
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const float2 x = S[k1 * kRrRow + i];
        r[i] = {x.x, x.y};
    }
    dft16<true>(r);
}

__device__ __forceinline__ void inv512_row(cx<float> *r, float2 *S, int k1, const float2 *__restrict__ tw)
{
    dft16<false>(r);
#pragma unroll
    for (int a = 1; a < 16; ++a) {
        const float2 q = tw[a * k1];
        r[a] = cmulc(r[a], cx<float>{q.x, q.y});
    }
#pragma unroll
    for (int a = 0; a < 16; ++a) S[k1 * kRrRow + a] = make_float2(r[a].re, r[a].im);
}

__device__ __forceinline__ void inv512_cols(cx<float> *v, const float2 *S, int t)
{
    __syncwarp();
#pragma unroll
    for (int k1 = 0; k1 < 32; ++k1) {
        const float2 x = S[k1 * kRrRow + t];
        v[k1] = {x.x, x.y};
    }
    dft32<false, false, true>(v);
}

// 16-byte asynchronous copy global -> shared (cp.async, completion by wait_group).
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Conv pass: one line of padded length 512 (n = 256 stored values) per 16 threads.
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
    cx<float> v[32];
#pragma unroll
    for (int m = 0; m < 16; ++m) {
        const float2 x = active ? w[t + 16 * m] : make_float2(0.f, 0.f);
        v[m] = {x.x, x.y};
    }
    fwd512_cols(v, S, t, tw);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int k1 = t + 16 * h;
        cx<float> *r = v + 16 * h;
        fwd512_row(r, S, k1);
#pragma unroll
        for (int k2 = 0; k2 < 16; ++k2) {
            const int k = k1 + 32 * k2;
            const float m = active ? mrow[full ? k : min(k, 512 - k)] : 0.f;
            r[k2] = {r[k2].re * m, r[k2].im * m};
        }
        inv512_row(r, S, k1, tw);
    }
    inv512_cols(v, S, t);
    if (active) {
#pragma unroll
        for (int b = 0; b < 16; ++b) w[t + 16 * b] = make_float2(v[b].re, v[b].im);
    }
}

// 3D y-forward pass, ny = 256 (My = 512): W1[z][kx][y] -> W2[kx][ky][z].  CTA
// (bx, kx) takes z = 16 bx .. 16 bx + 15; the outputs go through shared memory
// (row ky of 16 z values, pitch 17) so that each ky row is written as 128
// contiguous bytes.  The staging buffer is the transpose buffers' space.
__global__ void __launch_bounds__(16 * kRrLinesPerCta, 2)
    k_yf_rr512(const float2 *__restrict__ W1, float2 *__restrict__ W2, int nz, int hx, const float2 *__restrict__ tw)
{
    extern __shared__ float2 sbuf[];
    const int t = threadIdx.x & 15;
    const int l = threadIdx.x >> 4;
    const int kx = blockIdx.y;
    const int z0 = blockIdx.x * kRrLinesPerCta;
    const int z = z0 + l;
    const bool active = z < nz;
    float2 *S = sbuf + l * kRrLineElems;
    const float2 *in = W1 + ((size_t)(active ? z : 0) * hx + kx) * 256;
    cx<float> v[32];
#pragma unroll
    for (int m = 0; m < 16; ++m) {
        const float2 x = active ? in[t + 16 * m] : make_float2(0.f, 0.f);
        v[m] = {x.x, x.y};
    }
    fwd512_cols(v, S, t, tw);
    fwd512_row(v, S, t);
    fwd512_row(v + 16, S, t + 16);
    __syncthreads();                      // every line done with its transpose buffer
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int k2 = 0; k2 < 16; ++k2) {
            const int k = t + 16 * h + 32 * k2;
            sbuf[k * kRrRow + l] = make_float2(v[16 * h + k2].re, v[16 * h + k2].im);
        }
    __syncthreads();
    float2 *out = W2 + (size_t)kx * 512 * nz;
    for (int i = threadIdx.x; i < 512 * 16; i += blockDim.x) {
        const int ky = i >> 4, zz = z0 + (i & 15);
        if (zz < nz) out[(size_t)ky * nz + zz] = sbuf[ky * kRrRow + (i & 15)];
    }
}

// 3D y-inverse pass, ny = 256: W2[kx][ky][z] -> W1[z][kx][y] (crop to y < 256).
// Tile (z-block zb, kx): the kRrYiLines z-lines z = kRrYiLines zb + 0.. at kx,
// whose input is 512 rows ky of kRrYiLines consecutive z (64 bytes each) in
// W2[kx].  Each CTA takes tiles blockIdx.x, blockIdx.x + gridDim.x, ...; the
// next tile's rows are copied with cp.async into a staging buffer (pitch 10
// elements: 16-byte aligned rows, two-way bank conflicts on the transposed
// read) while the current tile is transformed.  Three CTAs of 4 warps fit an SM.
constexpr int kRrYiLines = 8;
constexpr int kRrStagePitch = 10;
constexpr size_t kRrYiSmem = sizeof(float2) * (kRrYiLines * kRrLineElems + 512 * kRrStagePitch);

__device__ __forceinline__ void yi_stage_tile(float2 *stage, const float2 *W2, int tile, int nzb, int nz)
{
    const int kx = tile / nzb, z0 = (tile - kx * nzb) * kRrYiLines;
    const float2 *in = W2 + (size_t)kx * 512 * nz;
    const int zv = min(kRrYiLines, nz - z0);
    if (zv == kRrYiLines && (nz % 2) == 0) {
        // whole 64-byte rows, 16 bytes (2 values) per copy
        for (int i = threadIdx.x; i < 512 * (kRrYiLines / 2); i += blockDim.x) {
            const int ky = i / (kRrYiLines / 2), c = i % (kRrYiLines / 2);
            cp_async16(stage + ky * kRrStagePitch + 2 * c, in + (size_t)ky * nz + z0 + 2 * c);
        }
    } else {
        // ragged z-block or odd row pitch: plain loads (zeros past nz)
        for (int i = threadIdx.x; i < 512 * kRrYiLines; i += blockDim.x) {
            const int ky = i / kRrYiLines, r = i % kRrYiLines, zz = z0 + r;
            stage[ky * kRrStagePitch + r] = zz < nz ? in[(size_t)ky * nz + zz] : make_float2(0.f, 0.f);
        }
    }
    cp_async_commit();
}

__global__ void __launch_bounds__(16 * kRrYiLines, 3)
    k_yi_rr512(const float2 *__restrict__ W2, float2 *__restrict__ W1, int nz, int hx, const float2 *__restrict__ tw)
{
    extern __shared__ float2 sbuf[];   // transpose buffers, then the staging buffer
    const int t = threadIdx.x & 15;
    const int l = threadIdx.x >> 4;
    float2 *S = sbuf + l * kRrLineElems;
    float2 *stage = sbuf + kRrYiLines * kRrLineElems;
    const int nzb = (nz + kRrYiLines - 1) / kRrYiLines;
    const int ntiles = nzb * hx;
    int tile = blockIdx.x;
    if (tile < ntiles) yi_stage_tile(stage, W2, tile, nzb, nz);
    for (; tile < ntiles; tile += gridDim.x) {
        const int kx = tile / nzb, z0 = (tile - kx * nzb) * kRrYiLines;
        const int z = z0 + l;
        cp_async_wait_all();
        __syncthreads();                  // the tile's rows are in the staging buffer
        cx<float> v[32];
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int k2 = 0; k2 < 16; ++k2) {
                const float2 x = stage[(t + 16 * h + 32 * k2) * kRrStagePitch + l];
                v[16 * h + k2] = {x.x, x.y};
            }
        __syncthreads();                  // staging buffer read: the next tile may land
        if (tile + (int)gridDim.x < ntiles) yi_stage_tile(stage, W2, tile + gridDim.x, nzb, nz);
        inv512_row(v, S, t, tw);
        inv512_row(v + 16, S, t + 16, tw);
        inv512_cols(v, S, t);
        if (z < nz) {
            float2 *out = W1 + ((size_t)z * hx + kx) * 256;
#pragma unroll
            for (int b = 0; b < 16; ++b) out[t + 16 * b] = make_float2(v[b].re, v[b].im);
        }
        __syncwarp();                     // the line's transpose buffer is free for the next tile
    }
    cp_async_wait_all();
}

// x passes, nx = 256 (Mx = 512): 8 complex lines (16 real rows) per CTA of 128
// threads.  Shared memory: the lines' transpose buffers, then the staging
// buffer of the transposed side W1[z][kx][y] (257 rows kx of 16 y, pitch 17).
constexpr int kRrXLines = 8;
constexpr int kRrXPitch = 17;
constexpr size_t kRrXSmem = sizeof(float2) * (kRrXLines * kRrLineElems + 257 * kRrXPitch);

// x forward: rows y, y + 1 of rho form one complex line Z; after the transform
// 2 A[k] = Z[k] + conj Z[-k], 2 B[k] = -i (Z[k] - conj Z[-k]) for k = 0..256
// (the factor 2 is removed by the multiplier), written to W1[z][k][y].
__global__ void __launch_bounds__(16 * kRrXLines, 3)
    k_xf_rr512(const float *__restrict__ rho, float2 *__restrict__ W1, int ny, const float2 *__restrict__ tw)
{
    extern __shared__ float2 sbuf[];
    const int t = threadIdx.x & 15;
    const int l = threadIdx.x >> 4;
    const int z = blockIdx.y;
    const int y0 = blockIdx.x * 2 * kRrXLines;
    const int ya = y0 + 2 * l;
    float2 *S = sbuf + l * kRrLineElems;
    float2 *T = sbuf + kRrXLines * kRrLineElems;
    const float *slab = rho + (size_t)z * ny * 256;
    cx<float> v[32];
#pragma unroll
    for (int m = 0; m < 16; ++m) {
        const float a = ya < ny ? slab[(size_t)ya * 256 + t + 16 * m] : 0.f;
        const float b = ya + 1 < ny ? slab[(size_t)(ya + 1) * 256 + t + 16 * m] : 0.f;
        v[m] = {a, b};
    }
    fwd512_cols(v, S, t, tw);
    fwd512_row(v, S, t);
    fwd512_row(v + 16, S, t + 16);
    __syncwarp();                          // rows read: the buffer takes Z in natural order
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int k2 = 0; k2 < 16; ++k2) S[t + 16 * h + 32 * k2] = make_float2(v[16 * h + k2].re, v[16 * h + k2].im);
    __syncwarp();
    for (int k = t; k <= 256; k += 16) {
        const float2 zk = S[k], zm = S[(512 - k) & 511];
        const cx<float> p = {zk.x, zk.y}, q = {zm.x, -zm.y};   // Z[k], conj Z[-k]
        const cx<float> A = cadd(p, q), B = cmul_negi(csub(p, q));
        T[k * kRrXPitch + 2 * l] = make_float2(A.re, A.im);
        T[k * kRrXPitch + 2 * l + 1] = make_float2(B.re, B.im);
    }
    __syncthreads();
    float2 *out = W1 + (size_t)z * 257 * ny;
    for (int i = threadIdx.x; i < 257 * 16; i += blockDim.x) {
        const int k = i >> 4, r = i & 15;
        if (y0 + r < ny) out[(size_t)k * ny + y0 + r] = T[k * kRrXPitch + r];
    }
}

// x inverse: Z[k] = A + i B, Z[512 - k] = conj A + i conj B (A, B real at k = 0
// and 256), inverse transform, real part to row y and imaginary part to row y + 1.
// Tile (y-block yb, z): rows y = 16 yb .. 16 yb + 15 of slab z, whose input is
// 257 rows k of 16 consecutive y (128 bytes each) in W1[z].  Each CTA takes
// tiles blockIdx.x, blockIdx.x + gridDim.x, ...; the next tile's rows are
// copied with cp.async into the staging buffer T (pitch 18 elements: 16-byte
// aligned rows) while the current tile is transformed.
constexpr int kRrXiPitch = 18;
constexpr size_t kRrXiSmem = sizeof(float2) * (kRrXLines * kRrLineElems + 257 * kRrXiPitch);

__device__ __forceinline__ void xi_stage_tile(float2 *T, const float2 *W1, int tile, int nyb, int ny)
{
    const int z = tile / nyb, y0 = (tile - z * nyb) * 2 * kRrXLines;
    const float2 *in = W1 + (size_t)z * 257 * ny;
    if (y0 + 2 * kRrXLines <= ny && (ny % 2) == 0) {
        // whole 128-byte rows, 16 bytes (2 values) per copy
        for (int i = threadIdx.x; i < 257 * kRrXLines; i += blockDim.x) {
            const int k = i / kRrXLines, c = i % kRrXLines;
            cp_async16(T + k * kRrXiPitch + 2 * c, in + (size_t)k * ny + y0 + 2 * c);
        }
    } else {
        // ragged y-block or odd row pitch: plain loads (zeros past ny)
        for (int i = threadIdx.x; i < 257 * 16; i += blockDim.x) {
            const int k = i >> 4, r = i & 15;
            T[k * kRrXiPitch + r] = y0 + r < ny ? in[(size_t)k * ny + y0 + r] : make_float2(0.f, 0.f);
        }
    }
    cp_async_commit();
}

__global__ void __launch_bounds__(16 * kRrXLines, 3)
    k_xi_rr512(const float2 *__restrict__ W1, float *__restrict__ u, int ny, int nz, const float2 *__restrict__ tw)
{
    extern __shared__ float2 sbuf[];
    const int t = threadIdx.x & 15;
    const int l = threadIdx.x >> 4;
    float2 *S = sbuf + l * kRrLineElems;
    float2 *T = sbuf + kRrXLines * kRrLineElems;
    const int nyb = (ny + 2 * kRrXLines - 1) / (2 * kRrXLines);
    const int ntiles = nyb * nz;
    int tile = blockIdx.x;
    if (tile < ntiles) xi_stage_tile(T, W1, tile, nyb, ny);
    for (; tile < ntiles; tile += gridDim.x) {
        const int z = tile / nyb, y0 = (tile - z * nyb) * 2 * kRrXLines;
        const int ya = y0 + 2 * l;
        cp_async_wait_all();
        __syncthreads();                       // the tile's rows are in T
        for (int k = t; k <= 256; k += 16) {
            const float2 a = T[k * kRrXiPitch + 2 * l], b = T[k * kRrXiPitch + 2 * l + 1];
            cx<float> A = {a.x, a.y}, B = {b.x, b.y};
            if (k == 0 || k == 256) {
                A.im = 0.f;
                B.im = 0.f;
            }
            const cx<float> zk = cadd(A, cmul_posi(B));
            S[k] = make_float2(zk.re, zk.im);
            if (k > 0 && k < 256) {
                const cx<float> zm = cadd(cconj(A), cmul_posi(cconj(B)));
                S[512 - k] = make_float2(zm.re, zm.im);
            }
        }
        __syncthreads();                       // T read: the next tile may land
        if (tile + (int)gridDim.x < ntiles) xi_stage_tile(T, W1, tile + gridDim.x, nyb, ny);
        cx<float> v[32];
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int k2 = 0; k2 < 16; ++k2) {
                const float2 x = S[t + 16 * h + 32 * k2];
                v[16 * h + k2] = {x.x, x.y};
            }
        __syncwarp();                          // natural order read: the buffer takes the rows
        inv512_row(v, S, t, tw);
        inv512_row(v + 16, S, t + 16, tw);
        inv512_cols(v, S, t);
        float *slab = u + (size_t)z * ny * 256;
        if (ya < ny) {
#pragma unroll
            for (int b = 0; b < 16; ++b) slab[(size_t)ya * 256 + t + 16 * b] = v[b].re;
        }
        if (ya + 1 < ny) {
#pragma unroll
            for (int b = 0; b < 16; ++b) slab[(size_t)(ya + 1) * 256 + t + 16 * b] = v[b].im;
        }
        __syncwarp();                          // the line's buffer is free for the next tile
    }
    cp_async_wait_all();
}

// Raise the kernel's dynamic shared-memory limit to kRrSmem once per device;
// `raised` is the kernel's own flag array (the kernels share a function type).
template <class K>
cudaError_t raise_rr(K kernel, bool *raised, size_t smem = kRrSmem)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64 && raised[dev]) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess && dev >= 0 && dev < 64) raised[dev] = true;
    return e;
}

}  // namespace

// Conv pass of an FP32 plan whose conv lines have padded length 512 (n = 256).
gsm_status_t launch_conv_rr512_f32(void *W, const void *mult, int nlines, int is3d, int My, int ny1, bool full,
                                   const void *tw, cudaStream_t st)
{
    static bool raised[64] = {};
    GSM_CUDA_TRY(raise_rr(k_conv_rr512, raised));
    const int blocks = (nlines + kRrLinesPerCta - 1) / kRrLinesPerCta;
    k_conv_rr512<<<blocks, 16 * kRrLinesPerCta, kRrSmem, st>>>(static_cast<float2 *>(W),
                                                               static_cast<const float *>(mult), nlines, is3d, My,
                                                               ny1, full ? 1 : 0, static_cast<const float2 *>(tw));
    return GSM_OK;   // a launch error stays pending for the caller's check
}

// y passes of a 3D FP32 plan with ny = 256: forward (W1 -> W2) or inverse (W2 -> W1).
gsm_status_t launch_y_rr512_f32(bool inverse, const void *in, void *out, int nz, int hx, const void *tw,
                                cudaStream_t st)
{
    dim3 g((nz + kRrLinesPerCta - 1) / kRrLinesPerCta, hx);
    if (!inverse) {
        static bool raised_f[64] = {};
        GSM_CUDA_TRY(raise_rr(k_yf_rr512, raised_f));
        k_yf_rr512<<<g, 16 * kRrLinesPerCta, kRrSmem, st>>>(static_cast<const float2 *>(in),
                                                            static_cast<float2 *>(out), nz, hx,
                                                            static_cast<const float2 *>(tw));
    } else {
        static bool raised_i[64] = {};
        static int resident[64] = {};
        GSM_CUDA_TRY(raise_rr(k_yi_rr512, raised_i, kRrYiSmem));
        int dev = 0;
        GSM_CUDA_TRY(cudaGetDevice(&dev));
        if (dev < 0 || dev >= 64) return GSM_ERR_INVALID_ARG;
        if (resident[dev] == 0) {
            int occ = 0, sms = 0;
            GSM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_yi_rr512, 16 * kRrYiLines,
                                                                       kRrYiSmem));
            GSM_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
            resident[dev] = std::max(1, occ) * sms;
        }
        const int tiles = ((nz + kRrYiLines - 1) / kRrYiLines) * hx;
        const int blocks = std::max(1, std::min(tiles, resident[dev]));
        k_yi_rr512<<<blocks, 16 * kRrYiLines, kRrYiSmem, st>>>(static_cast<const float2 *>(in),
                                                                   static_cast<float2 *>(out), nz, hx,
                                                                   static_cast<const float2 *>(tw));
    }
    return GSM_OK;   // a launch error stays pending for the caller's check
}

// x passes of an FP32 plan with nx = 256 on the z-slabs [0, nz): forward
// (rho -> W1) or inverse (W1 -> u); the pointers are those of slab 0.
gsm_status_t launch_x_rr512_f32(bool inverse, const void *in, void *out, int ny, int nz, const void *tw,
                                cudaStream_t st)
{
    dim3 g((ny + 2 * kRrXLines - 1) / (2 * kRrXLines), nz);
    if (!inverse) {
        static bool raised_f[64] = {};
        GSM_CUDA_TRY(raise_rr(k_xf_rr512, raised_f, kRrXSmem));
        k_xf_rr512<<<g, 16 * kRrXLines, kRrXSmem, st>>>(static_cast<const float *>(in), static_cast<float2 *>(out),
                                                        ny, static_cast<const float2 *>(tw));
    } else {
        static bool raised_i[64] = {};
        static int resident[64] = {};
        GSM_CUDA_TRY(raise_rr(k_xi_rr512, raised_i, kRrXiSmem));
        int dev = 0;
        GSM_CUDA_TRY(cudaGetDevice(&dev));
        if (dev < 0 || dev >= 64) return GSM_ERR_INVALID_ARG;
        if (resident[dev] == 0) {
            int occ = 0, sms = 0;
            GSM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_xi_rr512, 16 * kRrXLines, kRrXiSmem));
            GSM_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
            resident[dev] = std::max(1, occ) * sms;
        }
        const int tiles = g.x * g.y;
        const int blocks = std::max(1, std::min(tiles, resident[dev]));
        k_xi_rr512<<<blocks, 16 * kRrXLines, kRrXiSmem, st>>>(static_cast<const float2 *>(in),
                                                              static_cast<float *>(out), ny, nz,
                                                              static_cast<const float2 *>(tw));
    }
    return GSM_OK;   // a launch error stays pending for the caller's check
}

}  // namespace gsm
