// gsm_passes.cu -- Algorithm 1, "Actual computation": the zero-padded FFT
// convolution with the stored multiplier (Eq. I1FFT with the Taylor
// correction of Sec. 2.3 folded in), for each precision.
//
// Data flow in 3D (n = grid points per axis, M = 2n the padded lengths,
// hx = nx + 1 the non-negative x frequencies of the real transform):
//   pass xf   rho[z][y][x]        -> W1[z][kx][y]      two real rows per complex
//                                                      line, length Mx, zero pad
//   pass yf   W1[z][kx][y]        -> W2[kx][ky][z]     length My, zero pad
//   pass conv W2[kx][ky][0..nz)   -> same, in place    length Mz: forward,
//                                                      multiply, inverse, crop
//   pass yi   W2[kx][ky][z]       -> W1[z][kx][y]      length My, crop
//   pass xi   W1[z][kx][y]        -> u[z][y][x]        Hermitian fill, crop
// Each pass reads contiguous lines or writes them, and does the transposition
// in shared memory; the other side of each pass moves chunks of 2nl (xf, xi)
// or nl (yf, yi) consecutive complex values.  In 2D: xf (one slab), conv on
// W[kx][y] along y, xi.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <new>
#include <string>
#include <vector>
#include <type_traits>

#include <cooperative_groups.h>
#include <cuda.h>

#include "gsm_internal.h"

namespace gsm {

namespace {

constexpr int kMaxThreads = 512;   // CTA size cap: leaves 128 registers per thread

template <class Pol>
using S_t = typename Pol::scplx;

// Read of workspace data.  CG = true (the batch queue kernel, in which the
// workspace is written and read again by other CTAs of the same launch): the
// load bypasses L1 and the read-only path (ld.global.cg), so it sees what
// other CTAs stored before they signalled completion.
template <bool CG, class T>
__device__ __forceinline__ T ldw(const T *p)
{
    if constexpr (CG) return __ldcg(p);
    else return *p;
}

// Copies `count` elements into shared memory with U global loads in flight
// per thread (all U loads are issued before the first store waits for its
// data): for i = t, t + T, ... < count, dst(i, src(i)).
template <int U, class Val, class Src, class Dst>
__device__ __forceinline__ void gather_smem(int t, int T, int count, Src src, Dst dst)
{
    for (int i0 = t; i0 < count; i0 += U * T) {
        Val v[U];
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (i0 + u * T < count) v[u] = src(i0 + u * T);
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (i0 + u * T < count) dst(i0 + u * T, v[u]);
    }
}
// Loads in flight per thread when the y passes and the x inverse gather their
// input: four in double-float, whose y and x inverse passes wait on their
// gathered rows (measured 0.61 -> 0.53 ms for the y inverse at 256^3); one
// in FP64 and FP32, where more did not pay.
template <class Pol>
constexpr int kGatherDepth = std::is_same<Pol, DF64>::value ? 4 : 1;

// FP64 twiddle tables hold, after the M twiddles w^m, the constants of the
// FMA-form radix-8 stages (fft_stage8_fma); the other precisions have none.
template <class Pol>
__device__ __forceinline__ const double *g8_table(const typename Pol::tw_t *tw, int M)
{
    if constexpr (std::is_same<Pol, F64>::value) return reinterpret_cast<const double *>(tw + M);
    else return nullptr;
}

// Launch shape (see PassCfg): a CTA holds nl lines; line l is transformed by
// group l of gthr threads (blockDim.x = nl * gthr).  Loads and stores that
// touch one line are done by its group; the transposed side of a pass is
// done by the whole CTA, with one __syncthreads between it and the FFTs.

// The double-float x and y kernels with 8 elements per thread are compiled
// for four resident CTAs of up to 256 threads per SM (a 64-register bound):
// more warps to hide their global-memory and barrier waits (measured at
// 256^3: x forward 0.27 -> 0.25 ms, y inverse 0.53 -> 0.49, x inverse 0.29 ->
// 0.25).  Their launch shapes keep to 256 threads.
template <class Pol>
constexpr int xy_max_threads(int emax) { return (std::is_same<Pol, DF64>::value && emax == 8) ? 256 : kMaxThreads; }
template <class Pol>
constexpr int xy_min_ctas(int emax) { return (std::is_same<Pol, DF64>::value && emax == 8) ? 4 : 1; }

// ------------------------------------------------------------------ pass xf
// Each pass is a __device__ body taking its tile (bx, by) explicitly, so that
// the single-plan kernels and the grouped batch kernels share it.
template <class Pol, int EMAX>
__device__ __forceinline__ void body_xf(const typename Pol::io_t *__restrict__ rho, S_t<Pol> *__restrict__ W1,
                                        int nx, int ny, int hx, const Sched &sc, int nl, int gthr,
                                        const typename Pol::tw_t *__restrict__ tw, int bx, int by,
                                        unsigned char *smem_raw)
{
    using R = typename Pol::real;
    const int M = sc.M, LS = line_stride<Pol>(M);
    const Group g = make_group(gthr, nl);
    const int l = threadIdx.x / gthr;
    S_t<Pol> *s = reinterpret_cast<S_t<Pol> *>(smem_raw) + l * LS;
    const int z = by;
    const int y0 = bx * 2 * nl;
    const int ya = y0 + 2 * l;
    const typename Pol::io_t *slab = rho + (size_t)z * ny * nx;
    // x >= nx is zero padding: written only when the first stage reads it
    for (int x = g.t; x < (Pol::kPrune ? nx : M); x += g.T) {
        R a = Pol::zero(), b = Pol::zero();
        if (x < nx) {
            if (ya < ny) a = Pol::from_io(slab[(size_t)ya * nx + x]);
            if (ya + 1 < ny) b = Pol::from_io(slab[(size_t)(ya + 1) * nx + x]);
        }
        s[pidx<Pol>(x)] = Pol::st(cx<R>{a, b});
    }
    group_sync(g);
    fft_line<Pol, true, EMAX, Pol::kPrune, false>(s, sc, tw, g, g8_table<Pol>(tw, M));
    __syncthreads();
    // Z = A + iB with A, B the transforms of the two real rows:
    // 2A[k] = Z[k] + conj Z[-k], 2B[k] = -i (Z[k] - conj Z[-k]); the factor 2
    // is removed by the multiplier.
    const S_t<Pol> *s0 = reinterpret_cast<const S_t<Pol> *>(smem_raw);
    S_t<Pol> *out = W1 + (size_t)z * hx * ny;
    for (int i = threadIdx.x; i < hx * nl; i += blockDim.x) {
        const int k = i / nl, ll = i - k * nl;
        const cx<R> zk = Pol::ld(s0[ll * LS + pidx<Pol>(k)]);
        const cx<R> zm = cconj(Pol::ld(s0[ll * LS + pidx<Pol>(k == 0 ? 0 : M - k)]));
        const int yy = y0 + 2 * ll;
        if (yy < ny) out[(size_t)k * ny + yy] = Pol::st(cadd(zk, zm));
        if (yy + 1 < ny) out[(size_t)k * ny + yy + 1] = Pol::st(cmul_negi(csub(zk, zm)));
    }
}

template <class Pol, int EMAX>
__global__ void __launch_bounds__(xy_max_threads<Pol>(EMAX), xy_min_ctas<Pol>(EMAX))
    k_xf(const typename Pol::io_t *__restrict__ rho, S_t<Pol> *__restrict__ W1, int nx, int ny, int hx,
         Sched sc, int nl, int gthr, const typename Pol::tw_t *__restrict__ tw)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    body_xf<Pol, EMAX>(rho, W1, nx, ny, hx, sc, nl, gthr, tw, blockIdx.x, blockIdx.y, smem_raw);
}

// ------------------------------------------------------------------ pass yf
template <class Pol, int EMAX, bool CG = false>
__device__ __forceinline__ void body_yf(const S_t<Pol> *__restrict__ W1, S_t<Pol> *__restrict__ W2, int ny,
                                        int nz, int hx, const Sched &sc, int nl, int gthr,
                                        const typename Pol::tw_t *__restrict__ tw, int bx, int by,
                                        unsigned char *smem_raw)
{
    using R = typename Pol::real;
    const int M = sc.M, LS = line_stride<Pol>(M);
    const Group g = make_group(gthr, nl);
    const int l = threadIdx.x / gthr;
    S_t<Pol> *s = reinterpret_cast<S_t<Pol> *>(smem_raw) + l * LS;
    const int kx = by;
    const int z0 = bx * nl;
    const int z = z0 + l;
    const S_t<Pol> *in = W1 + ((size_t)z * hx + kx) * ny;
    gather_smem<kGatherDepth<Pol>, S_t<Pol>>(   // y >= ny: zero padding
        g.t, g.T, Pol::kPrune ? ny : M,
        [&](int y) {
            S_t<Pol> v = Pol::st(cx<R>{Pol::zero(), Pol::zero()});
            if (y < ny && z < nz) v = ldw<CG>(in + y);
            return v;
        },
        [&](int y, const S_t<Pol> &v) { s[pidx<Pol>(y)] = v; });
    group_sync(g);
    fft_line<Pol, true, EMAX, Pol::kPrune, false>(s, sc, tw, g, g8_table<Pol>(tw, M));
    __syncthreads();
    const S_t<Pol> *s0 = reinterpret_cast<const S_t<Pol> *>(smem_raw);
    S_t<Pol> *out = W2 + (size_t)kx * M * nz;
    for (int i = threadIdx.x; i < M * nl; i += blockDim.x) {
        const int ky = i / nl, ll = i - ky * nl;
        const int zz = z0 + ll;
        if (zz < nz) out[(size_t)ky * nz + zz] = s0[ll * LS + pidx<Pol>(ky)];
    }
}

template <class Pol, int EMAX>
__global__ void __launch_bounds__(xy_max_threads<Pol>(EMAX), xy_min_ctas<Pol>(EMAX))
    k_yf(const S_t<Pol> *__restrict__ W1, S_t<Pol> *__restrict__ W2, int ny, int nz, int hx, Sched sc,
         int nl, int gthr, const typename Pol::tw_t *__restrict__ tw)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    body_yf<Pol, EMAX>(W1, W2, ny, nz, hx, sc, nl, gthr, tw, blockIdx.x, blockIdx.y, smem_raw);
}

// ------------------------------------------------------------------ pass conv
// Lines of length n (stored) padded to M: forward, multiply by the real
// multiplier mult[row + min(k, M - k)], inverse, keep the first n.
// 3D: line = kx * My + ky, row = (kx * (ny + 1) + min(ky, My - ky)) * (nz + 1).
// 2D: line = kx, row = kx * (ny + 1).  Entirely group-local: no CTA barrier.
// full: the multiplier is stored for the whole half spectrum, row line * M.
template <class Pol, int EMAX, bool CG = false>
__device__ __forceinline__ void body_conv(S_t<Pol> *__restrict__ W, const typename Pol::mult_t *__restrict__ mult,
                                          int nlines, int n, int is3d, int My, int ny1, const Sched &sc,
                                          const Sched &sci, int nl, int gthr,
                                          const typename Pol::tw_t *__restrict__ tw,
                                          const typename Pol::tw_t *__restrict__ twi, int bx,
                                          unsigned char *smem_raw, bool full = false)
{
    using R = typename Pol::real;
    const int M = sc.M, LS = line_stride<Pol>(M);
    const Group g = make_group(gthr, nl);
    const int l = threadIdx.x / gthr;
    S_t<Pol> *s = reinterpret_cast<S_t<Pol> *>(smem_raw) + l * LS;
    const int line = bx * nl + l;
    if (line >= nlines) return;   // the whole group leaves; no CTA barrier follows
    S_t<Pol> *w = W + (size_t)line * n;
    for (int z = g.t; z < (Pol::kPruneConv ? n : M); z += g.T) {   // z >= n: zero padding
        S_t<Pol> v = Pol::st(cx<R>{Pol::zero(), Pol::zero()});
        if (z < n) v = ldw<CG>(w + z);
        s[pidx<Pol>(z)] = v;
    }
    group_sync(g);
    // multiplier of frequency k: the whole half spectrum is stored (full), or
    // the octant, read at min(k, M - k) (the multiplier is even)
    const typename Pol::mult_t *mrow;
    if (full) {
        mrow = mult + (size_t)line * M;
    } else if (is3d) {
        const int kx = line / My, ky = line - kx * My;
        mrow = mult + ((size_t)kx * ny1 + min(ky, My - ky)) * (n + 1);
    } else {
        mrow = mult + (size_t)line * (n + 1);
    }
    auto mult_of = [&](int k) -> R { return Pol::mult(mrow[full ? k : min(k, M - k)]); };
    const double *gt = g8_table<Pol>(tw, M), *gti = g8_table<Pol>(twi, M);
    const int fr = fused_radix(sc, sci);
    if (fr != 0) {
        // forward up to its last stage; last forward stage, multiplication and
        // first inverse stage in registers; the rest of the inverse
        fft_line<Pol, true, EMAX, Pol::kPruneConv, false>(s, sc, tw, g, gt, 0, sc.nst - 1);
        if (fr == 8) fft_fused_mid<Pol, 8, (EMAX + 7) / 8>(s, sc, tw, g, gt, mult_of);
        else if (fr == 4) fft_fused_mid<Pol, 4, (EMAX + 3) / 4>(s, sc, tw, g, gt, mult_of);
        else if (fr == 2) fft_fused_mid<Pol, 2, (EMAX + 1) / 2>(s, sc, tw, g, gt, mult_of);
        else if (fr == 5) fft_fused_mid<Pol, 5, (EMAX + 4) / 5>(s, sc, tw, g, gt, mult_of);
        else fft_fused_mid<Pol, 3, (EMAX + 2) / 3>(s, sc, tw, g, gt, mult_of);
        fft_line<Pol, false, EMAX, false, Pol::kPruneConv>(s, sci, twi, g, gti, 1);
    } else {
        fft_line<Pol, true, EMAX, Pol::kPruneConv, false>(s, sc, tw, g, gt);
        for (int k = g.t; k < M; k += g.T) {
            const int p = pidx<Pol>(k);
            s[p] = Pol::st(cscale(Pol::ld(s[p]), mult_of(k)));
        }
        group_sync(g);
        fft_line<Pol, false, EMAX, false, Pol::kPruneConv>(s, sci, twi, g, gti);
    }
    for (int z = g.t; z < n; z += g.T) w[z] = s[pidx<Pol>(z)];
}

// The double-float conv kernel with 8 elements per thread is compiled for
// three resident CTAs of up to 256 threads per SM (an 85-register bound):
// more warps to hide its stalls than at its natural 108 registers (measured
// 1.54 -> 1.50 ms at 256^3).  Its launch shapes keep to 256 threads.
template <class Pol>
constexpr int conv_max_threads(int emax) { return (std::is_same<Pol, DF64>::value && emax == 8) ? 256 : kMaxThreads; }
template <class Pol>
constexpr int conv_min_ctas(int emax) { return (std::is_same<Pol, DF64>::value && emax == 8) ? 3 : 1; }

template <class Pol, int EMAX>
__global__ void __launch_bounds__(conv_max_threads<Pol>(EMAX), conv_min_ctas<Pol>(EMAX))
    k_conv(S_t<Pol> *__restrict__ W, const typename Pol::mult_t *__restrict__ mult,
                                                      int nlines, int n, int is3d, int My, int ny1, Sched sc,
                                                      Sched sci, int nl, int gthr,
                                                      const typename Pol::tw_t *__restrict__ tw,
                                                      const typename Pol::tw_t *__restrict__ twi, int full)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    body_conv<Pol, EMAX>(W, mult, nlines, n, is3d, My, ny1, sc, sci, nl, gthr, tw, twi, blockIdx.x, smem_raw,
                         full != 0);
}

// ------------------------------------------------------------------ pass yi
template <class Pol, int EMAX, bool CG = false>
__device__ __forceinline__ void body_yi(const S_t<Pol> *__restrict__ W2, S_t<Pol> *__restrict__ W1, int ny,
                                        int nz, int hx, const Sched &sc, int nl, int gthr,
                                        const typename Pol::tw_t *__restrict__ tw, int bx, int by,
                                        unsigned char *smem_raw)
{
    const int M = sc.M, LS = line_stride<Pol>(M);
    const Group g = make_group(gthr, nl);
    const int l = threadIdx.x / gthr;
    S_t<Pol> *s0 = reinterpret_cast<S_t<Pol> *>(smem_raw);
    S_t<Pol> *s = s0 + l * LS;
    const int kx = by;
    const int z0 = bx * nl;
    const S_t<Pol> *in = W2 + (size_t)kx * M * nz;
    gather_smem<kGatherDepth<Pol>, S_t<Pol>>(
        threadIdx.x, blockDim.x, M * nl,
        [&](int i) {
            const int ky = i / nl, ll = i - ky * nl;
            S_t<Pol> v{};
            if (z0 + ll < nz) v = ldw<CG>(in + (size_t)ky * nz + z0 + ll);
            return v;
        },
        [&](int i, const S_t<Pol> &v) {
            const int ky = i / nl, ll = i - ky * nl;
            if (z0 + ll < nz) s0[ll * LS + pidx<Pol>(ky)] = v;
        });
    __syncthreads();
    const int z = z0 + l;
    fft_line<Pol, false, EMAX, false, Pol::kPrune>(s, sc, tw, g, g8_table<Pol>(tw, M));
    if (z < nz) {
        S_t<Pol> *out = W1 + ((size_t)z * hx + kx) * ny;
        for (int y = g.t; y < ny; y += g.T) out[y] = s[pidx<Pol>(y)];
    }
}

template <class Pol, int EMAX>
__global__ void __launch_bounds__(xy_max_threads<Pol>(EMAX), xy_min_ctas<Pol>(EMAX))
    k_yi(const S_t<Pol> *__restrict__ W2, S_t<Pol> *__restrict__ W1, int ny, int nz, int hx, Sched sc,
         int nl, int gthr, const typename Pol::tw_t *__restrict__ tw)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    body_yi<Pol, EMAX>(W2, W1, ny, nz, hx, sc, nl, gthr, tw, blockIdx.x, blockIdx.y, smem_raw);
}

// ------------------------------------------------------------------ pass xi
template <class Pol, int EMAX, bool CG = false>
__device__ __forceinline__ void body_xi(const S_t<Pol> *__restrict__ W1, typename Pol::io_t *__restrict__ u, int nx,
                                        int ny, int hx, const Sched &sc, int nl, int gthr,
                                        const typename Pol::tw_t *__restrict__ tw, int bx, int by,
                                        unsigned char *smem_raw)
{
    using R = typename Pol::real;
    const int M = sc.M, LS = line_stride<Pol>(M);
    const Group g = make_group(gthr, nl);
    const int l = threadIdx.x / gthr;
    S_t<Pol> *s0 = reinterpret_cast<S_t<Pol> *>(smem_raw);
    S_t<Pol> *s = s0 + l * LS;
    const int z = by;
    const int y0 = bx * 2 * nl;
    const S_t<Pol> *in = W1 + (size_t)z * hx * ny;
    // Z[k] = A[k] + i B[k] (k = 0..nx), Z[M-k] = conj A[k] + i conj B[k];
    // A, B real at k = 0 and k = nx (DC and Nyquist of real rows)
    struct AB {
        S_t<Pol> a, b;
    };
    gather_smem<kGatherDepth<Pol>, AB>(
        threadIdx.x, blockDim.x, hx * nl,
        [&](int i) {
            const int k = i / nl, ll = i - k * nl;
            const int yy = y0 + 2 * ll;
            AB v{Pol::st(cx<R>{Pol::zero(), Pol::zero()}), Pol::st(cx<R>{Pol::zero(), Pol::zero()})};
            if (yy < ny) v.a = ldw<CG>(in + (size_t)k * ny + yy);
            if (yy + 1 < ny) v.b = ldw<CG>(in + (size_t)k * ny + yy + 1);
            return v;
        },
        [&](int i, const AB &v) {
            const int k = i / nl, ll = i - k * nl;
            cx<R> A = Pol::ld(v.a), B = Pol::ld(v.b);
            if (k == 0 || k == nx) {
                A.im = Pol::zero();
                B.im = Pol::zero();
            }
            s0[ll * LS + pidx<Pol>(k)] = Pol::st(cadd(A, cmul_posi(B)));
            if (k > 0 && k < nx) s0[ll * LS + pidx<Pol>(M - k)] = Pol::st(cadd(cconj(A), cmul_posi(cconj(B))));
        });
    __syncthreads();
    fft_line<Pol, false, EMAX, false, Pol::kPrune>(s, sc, tw, g, g8_table<Pol>(tw, M));
    const int ya = y0 + 2 * l;
    typename Pol::io_t *slab = u + (size_t)z * ny * nx;
    for (int x = g.t; x < nx; x += g.T) {
        const cx<R> c = Pol::ld(s[pidx<Pol>(x)]);
        if (ya < ny) slab[(size_t)ya * nx + x] = Pol::to_io(c.re);
        if (ya + 1 < ny) slab[(size_t)(ya + 1) * nx + x] = Pol::to_io(c.im);
    }
}

template <class Pol, int EMAX>
__global__ void __launch_bounds__(xy_max_threads<Pol>(EMAX), xy_min_ctas<Pol>(EMAX))
    k_xi(const S_t<Pol> *__restrict__ W1, typename Pol::io_t *__restrict__ u, int nx, int ny, int hx,
         Sched sc, int nl, int gthr, const typename Pol::tw_t *__restrict__ tw)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    body_xi<Pol, EMAX>(W1, u, nx, ny, hx, sc, nl, gthr, tw, blockIdx.x, blockIdx.y, smem_raw);
}

// ------------------------------------------------------------------ pass conv, long 2D lines
// A conv line of padded length M = 2 Mh holds Mh values x[0..Mh) and zeros.
// Its even and odd frequencies are then two transforms of length Mh:
//   X[2k] = FFT_Mh(x)[k],   X[2k + 1] = FFT_Mh(x w_M^n)[k],
// and the cropped inverse (outputs n < Mh) is
//   u[n] = IFFT_Mh(E)[n] + w_M^(-n) IFFT_Mh(O)[n],
// E, O the multiplied even and odd frequencies.  A cluster of two CTAs takes
// one line: rank 0 the even half, rank 1 the odd half (a line of Mh values
// each, half the shared memory of the whole line), then each adds its half of
// the outputs to the other CTA's through distributed shared memory.  Two CTAs
// per SM work on different lines, so one line's barrier-separated phases
// overlap another's (one CTA per SM held a whole line of 8192 and left the
// FP64 pipe idle during its shared-memory phases).  Schedules, tables:
// length Mh (sched_hf, sched_hi, twh, twhi); twM: the M twiddles w_M^m.
// A half line (at most 4096 values) takes at most 256 threads.  Three CTAs per
// SM in FP64 and double-float (an 80-register cap: their butterfly arrays
// partly spill, to L1) overlap the barrier-separated stages better than two:
// measured 4.17 -> 4.16 ms (FP64) and 1.41 -> 1.34 ms (FP32x2) for the conv at
// 4096^2.  FP32 keeps the engine's usual bound (a 256-thread bound made its
// conv slower, 0.50 -> 0.53 ms, with or without the three CTAs).
constexpr int kSplitThreads = 256;
template <class Pol>
constexpr int kSplitBoundThreads = std::is_same<Pol, F32>::value ? kMaxThreads : kSplitThreads;
template <class Pol>
constexpr int kSplitCtasPerSm = std::is_same<Pol, F32>::value ? 1 : 3;

template <class Pol, int EMAX>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kSplitBoundThreads<Pol>, kSplitCtasPerSm<Pol>)
    k_conv_split(S_t<Pol> *__restrict__ W, const typename Pol::mult_t *__restrict__ mult, int nlines, int ny1,
                 Sched sc, Sched sci, const typename Pol::tw_t *__restrict__ tw,
                 const typename Pol::tw_t *__restrict__ twi, const typename Pol::tw_t *__restrict__ twM, int full)
{
    using R = typename Pol::real;
    namespace cg = cooperative_groups;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int line = blockIdx.x >> 1;
    const int Mh = sc.M, M = 2 * Mh;
    const Group g = make_group(blockDim.x, 1);
    S_t<Pol> *s = reinterpret_cast<S_t<Pol> *>(smem_raw);
    S_t<Pol> *w = W + (size_t)line * Mh;
    const bool active = line < nlines;   // every CTA of a cluster reaches both cluster barriers
    if (active) {
        for (int i = g.t; i < Mh; i += g.T) {
            cx<R> v = Pol::ld(w[i]);
            if (rank) v = cmul(v, Pol::tw(twM[i]));   // x w_M^n
            s[pidx<Pol>(i)] = Pol::st(v);
        }
        group_sync(g);
        const typename Pol::mult_t *mrow = mult + (size_t)line * (full ? M : ny1);
        // output k' of this half is frequency k = 2 k' + rank
        auto mult_of = [&](int kk) -> R {
            const int k = 2 * kk + rank;
            return Pol::mult(mrow[full ? k : min(k, M - k)]);
        };
        const double *gt = g8_table<Pol>(tw, Mh), *gti = g8_table<Pol>(twi, Mh);
        const int fr = fused_radix(sc, sci);
        if (fr != 0) {
            fft_line<Pol, true, EMAX>(s, sc, tw, g, gt, 0, sc.nst - 1);
            if (fr == 8) fft_fused_mid<Pol, 8, (EMAX + 7) / 8>(s, sc, tw, g, gt, mult_of);
            else if (fr == 4) fft_fused_mid<Pol, 4, (EMAX + 3) / 4>(s, sc, tw, g, gt, mult_of);
            else if (fr == 2) fft_fused_mid<Pol, 2, (EMAX + 1) / 2>(s, sc, tw, g, gt, mult_of);
            else if (fr == 5) fft_fused_mid<Pol, 5, (EMAX + 4) / 5>(s, sc, tw, g, gt, mult_of);
            else fft_fused_mid<Pol, 3, (EMAX + 2) / 3>(s, sc, tw, g, gt, mult_of);
            fft_line<Pol, false, EMAX>(s, sci, twi, g, gti, 1);
        } else {
            fft_line<Pol, true, EMAX>(s, sc, tw, g, gt);
            for (int k = g.t; k < Mh; k += g.T) {
                const int p = pidx<Pol>(k);
                s[p] = Pol::st(cscale(Pol::ld(s[p]), mult_of(k)));
            }
            group_sync(g);
            fft_line<Pol, false, EMAX>(s, sci, twi, g, gti);
        }
        if (rank) {
            for (int i = g.t; i < Mh; i += g.T) {
                const int p = pidx<Pol>(i);
                s[p] = Pol::st(cmulc(Pol::ld(s[p]), Pol::tw(twM[i])));   // w_M^(-n)
            }
        }
    }
    cl.sync();   // both halves transformed
    if (active) {
        const S_t<Pol> *peer = cl.map_shared_rank(s, rank ^ 1);
        const int h = Mh / 2, n0 = rank * h;
        for (int i = g.t; i < h; i += g.T) {
            const int n = n0 + i, p = pidx<Pol>(n);
            w[n] = Pol::st(cadd(Pol::ld(s[p]), Pol::ld(peer[p])));
        }
    }
    cl.sync();   // the peer has read this CTA's half: its shared memory may go
}

// ------------------------------------------------------------------ x forward, long 2D lines
// An x line of padded length M = 2 Mh (two real rows as one complex line)
// holds Mh = nx values and zeros, so, as for the split conv, its even and odd
// frequencies are two transforms of length Mh, of x and of x w_M^n.  The
// forward needs no exchange: the Hermitian split pairs Z[k] with Z[M - k],
// which has the parity of k, so each CTA of a pair (rank = blockIdx.x & 1)
// transforms its half and writes the frequencies k = 2 k' + rank itself.
// Two lines of Mh per SM overlap each other's barrier-separated phases, where
// one line of 2 Mh per CTA filled an SM alone.  (The x inverse stays one line
// per CTA: split the same way, with the halves summed through distributed
// shared memory as in the conv, it was no faster, 1.19 -> 1.21 ms in FP64 at
// 4096^2; split by output parity, each CTA reading the whole half spectrum and
// writing every other output, it was slower, 1.19 -> 1.27 ms.)  sc: length
// Mh; tw: its tables; twM: the M twiddles w_M^m.
template <class Pol, int EMAX>
__global__ void __launch_bounds__(kSplitBoundThreads<Pol>, kSplitCtasPerSm<Pol>)
    k_xf_split(const typename Pol::io_t *__restrict__ rho, S_t<Pol> *__restrict__ W1, int nx, int ny, int hx,
               Sched sc, const typename Pol::tw_t *__restrict__ tw, const typename Pol::tw_t *__restrict__ twM)
{
    using R = typename Pol::real;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int rank = blockIdx.x & 1, ya = 2 * (blockIdx.x >> 1);
    const int Mh = sc.M;   // == nx
    const Group g = make_group(blockDim.x, 1);
    S_t<Pol> *s = reinterpret_cast<S_t<Pol> *>(smem_raw);
    for (int x = g.t; x < nx; x += g.T) {
        R a = Pol::zero(), b = Pol::zero();
        if (ya < ny) a = Pol::from_io(rho[(size_t)ya * nx + x]);
        if (ya + 1 < ny) b = Pol::from_io(rho[(size_t)(ya + 1) * nx + x]);
        cx<R> v{a, b};
        if (rank) v = cmul(v, Pol::tw(twM[x]));   // x w_M^x: the odd frequencies
        s[pidx<Pol>(x)] = Pol::st(v);
    }
    group_sync(g);
    fft_line<Pol, true, EMAX>(s, sc, tw, g, g8_table<Pol>(tw, Mh));
    // frequency k = 2 k' + rank sits at k' of this half; M - k at (Mh - k' - rank) mod Mh
    const int nk = rank ? nx / 2 : nx / 2 + 1;   // k = 0 .. nx of this parity (nx is even)
    for (int kp = threadIdx.x; kp < nk; kp += blockDim.x) {
        const int k = 2 * kp + rank;
        int km = Mh - kp - rank;
        if (km == Mh) km = 0;
        const cx<R> zk = Pol::ld(s[pidx<Pol>(kp)]);
        const cx<R> zm = cconj(Pol::ld(s[pidx<Pol>(km)]));
        if (ya < ny) W1[(size_t)k * ny + ya] = Pol::st(cadd(zk, zm));
        if (ya + 1 < ny) W1[(size_t)k * ny + ya + 1] = Pol::st(cmul_negi(csub(zk, zm)));
    }
}

// ------------------------------------------------------------------ FFT test hook
template <class Pol, bool FWD, int EMAX>
__global__ void __launch_bounds__(kMaxThreads) k_fft_hook(const double2 *__restrict__ in, double2 *__restrict__ out,
                                                          int nlines, Sched sc, int nl, int gthr,
                                                          const typename Pol::tw_t *__restrict__ tw, int use_g8)
{
    using R = typename Pol::real;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int M = sc.M, LS = line_stride<Pol>(M);
    const Group g = make_group(gthr, nl);
    const int l = threadIdx.x / gthr;
    S_t<Pol> *s = reinterpret_cast<S_t<Pol> *>(smem_raw) + l * LS;
    const int line = blockIdx.x * nl + l;
    if (line >= nlines) return;
    for (int k = g.t; k < M; k += g.T) {
        const double2 v = in[(size_t)line * M + k];
        s[pidx<Pol>(k)] = Pol::st(cx<R>{Pol::from_io((typename Pol::io_t)v.x), Pol::from_io((typename Pol::io_t)v.y)});
    }
    group_sync(g);
    fft_line<Pol, FWD, EMAX>(s, sc, tw, g, use_g8 ? g8_table<Pol>(tw, M) : nullptr);
    for (int k = g.t; k < M; k += g.T) {
        const cx<R> c = Pol::ld(s[pidx<Pol>(k)]);
        out[(size_t)line * M + k] = make_double2((double)Pol::to_io(c.re), (double)Pol::to_io(c.im));
    }
}

// ------------------------------------------------------------------ batch: one launch, a device work queue
// One launch applies up to kBatchMax plans of different sizes (one precision,
// one dimension).  The work is a queue of items (pass, instance, tile), a
// tile being one CTA's share of that instance's pass grid, in pass-major
// order: every item of pass p comes before every item of pass p + 1.  The
// launch has one CTA per item.  When a CTA starts, its thread 0 takes a ticket
// from an atomic counter (so items go to CTAs in the order the CTAs start,
// whatever their block index), waits until the instance's previous pass is
// complete (a counter of finished tiles per instance and pass), the CTA runs
// the tile with the same pass bodies as the single-plan kernels, and counts it
// as finished.  Each item's dependencies were taken earlier, by CTAs that are
// already resident and whose own dependencies were taken earlier still, so
// the waits always end, however many CTAs are resident.  Passes of different
// instances overlap and no launch boundary drains the GPU between passes.
// Each wait is bounded all the same: when it runs out the CTA records
// GSM_ERR_TIMEOUT in the status word and raises the abort flag, and every
// later CTA returns at once.  Every line is done by one warp holding up to 16
// elements per thread (M <= 512), nl lines per CTA, so one CTA shape serves
// all sizes and passes.  (A loop over items inside long-lived CTAs was tried
// first: with the pass bodies inside a loop the compiler no longer kept their
// butterfly arrays in registers, 3 to 13 KB of stack per thread.)
constexpr int kBatchMax = 48;
constexpr int kBatchEmax = 16;
constexpr int kBatchMaxM = 32 * kBatchEmax;
constexpr int kBatchPasses = 5;

struct InstDesc {
    const void *rho;
    void *u;
    void *W1, *W2;
    const void *mult;
    const void *tw[3], *twi[3];   // forward and inverse tables per axis
    int n[3], M[3];
    Sched sc[3], sci[3];          // forward and inverse schedules per axis
    int gx[kBatchPasses];   // x extent of each pass's tile grid
    int full;               // multiplier over the whole half spectrum
};

// Queue state of one launch in device memory, zeroed before the launch: the
// next item, the status word (0 or GSM_ERR_TIMEOUT), the abort flag, one
// unused word, then the finished-tile counter of each (instance, pass).
constexpr int kStateHeader = 4;
constexpr int kStateWords = kStateHeader + kBatchMax * kBatchPasses;

struct QueueArgs {
    int count, d, nl, npass;
    int total;                                  // items in the queue
    int start[kBatchPasses + 1];                // first item of each pass
    int tiles[kBatchPasses][kBatchMax + 1];     // within a pass: first tile of each instance
    unsigned *state;                            // kStateWords words
    unsigned long long wait_ns;                 // bound of every wait
    int hold;                                   // test hook: this instance's first pass never
                                                // counts as complete (-1: none)
    InstDesc inst[kBatchMax];
};

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned ld_relaxed_gpu(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Thread 0 of the CTA: take the next item and wait for its dependency.
// Returns false when the queue is empty, the batch was aborted or the wait ran
// out; otherwise the item's pass, instance and tile.
__device__ __forceinline__ bool take_item(const QueueArgs &a, int *pass, int *inst, int *tile)
{
    unsigned *next = a.state, *status = a.state + 1, *abort_flag = a.state + 2;
    const unsigned *done = a.state + kStateHeader;
    if (ld_relaxed_gpu(abort_flag) != 0) return false;
    const int item = (int)atomicAdd(next, 1u);
    if (item >= a.total) return false;
    int p = 0;
    while (item >= a.start[p + 1]) ++p;
    const int r = item - a.start[p];
    int i = 0;
    while (r >= a.tiles[p][i + 1]) ++i;
    *pass = p;
    *inst = i;
    *tile = r - a.tiles[p][i];
    if (p == 0) return true;
    const unsigned need = (unsigned)(a.tiles[p - 1][i + 1] - a.tiles[p - 1][i]) + (p == 1 && i == a.hold ? 1u : 0u);
    const unsigned *cnt = done + i * kBatchPasses + (p - 1);
    if (ld_acquire_gpu(cnt) >= need) return true;
    const unsigned long long t0 = global_ns();
    unsigned sleep_ns = 32;
    while (ld_acquire_gpu(cnt) < need) {
        if (ld_relaxed_gpu(abort_flag) != 0) return false;
        if (global_ns() - t0 > a.wait_ns) {
            atomicExch(status, (unsigned)GSM_ERR_TIMEOUT);
            atomicExch(abort_flag, 1u);
            return false;
        }
        __nanosleep(sleep_ns);
        if (sleep_ns < 1024) sleep_ns *= 2;
    }
    return true;
}

// One tile of pass PASS of one instance.
template <class Pol, int D, int PASS>
__device__ __forceinline__ void queue_tile(const InstDesc &d, int nl, int t, unsigned char *smem_raw)
{
    using io = typename Pol::io_t;
    using tw = typename Pol::tw_t;
    constexpr int last = D == 3 ? 4 : 2;
    const int gx = d.gx[PASS];
    const int bx = t % gx, by = t / gx;
    const int nx = d.n[0], ny = d.n[1], nz = D == 3 ? d.n[2] : 1, hx = nx + 1;
    S_t<Pol> *W1 = static_cast<S_t<Pol> *>(d.W1);
    S_t<Pol> *W2 = static_cast<S_t<Pol> *>(d.W2);
    const auto *mult = static_cast<const typename Pol::mult_t *>(d.mult);
    auto T = [&](const void *t) { return static_cast<const tw *>(t); };
    if constexpr (PASS == 0) {
        body_xf<Pol, kBatchEmax>(static_cast<const io *>(d.rho), W1, nx, ny, hx, d.sc[0], nl, 32, T(d.tw[0]), bx,
                                 by, smem_raw);
    } else if constexpr (PASS == last) {
        body_xi<Pol, kBatchEmax, true>(W1, static_cast<io *>(d.u), nx, ny, hx, d.sci[0], nl, 32, T(d.twi[0]), bx,
                                       by, smem_raw);
    } else if constexpr (D == 2) {
        body_conv<Pol, kBatchEmax, true>(W1, mult, hx, ny, 0, 1, ny + 1, d.sc[1], d.sci[1], nl, 32, T(d.tw[1]),
                                         T(d.twi[1]), bx, smem_raw, d.full != 0);
    } else if constexpr (PASS == 1) {
        body_yf<Pol, kBatchEmax, true>(W1, W2, ny, nz, hx, d.sc[1], nl, 32, T(d.tw[1]), bx, by, smem_raw);
    } else if constexpr (PASS == 2) {
        body_conv<Pol, kBatchEmax, true>(W2, mult, hx * d.M[1], nz, 1, d.M[1], ny + 1, d.sc[2], d.sci[2], nl, 32,
                                         T(d.tw[2]), T(d.twi[2]), bx, smem_raw, d.full != 0);
    } else {
        body_yi<Pol, kBatchEmax, true>(W2, W1, ny, nz, hx, d.sci[1], nl, 32, T(d.twi[1]), bx, by, smem_raw);
    }
}

// Item of a CTA (shared): valid if go != 0.
struct QueueItem {
    int go, pass, inst, tile;
};

// The tile of pass PASS if the CTA's item belongs to that pass, then one
// release of the instance's count for the pass.
template <class Pol, int D, int PASS>
__device__ __forceinline__ void queue_pass(const QueueArgs &a, const QueueItem &it, unsigned char *smem_raw)
{
    if (it.go && it.pass == PASS) {
        const int i = it.inst;
        queue_tile<Pol, D, PASS>(a.inst[i], a.nl, it.tile, smem_raw);
        // every thread's stores of the tile, then one release of the count
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned *cnt = a.state + kStateHeader + i * kBatchPasses + PASS;
            asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(cnt) : "memory");
        }
    }
}

template <class Pol, int D>
// Resident CTAs per SM asked of the compiler: FP64 and double-float 2 (a
// 128-register cap), FP32 5 (51 registers; its tiles are short, and more
// resident CTAs cover their ticket and acquire: measured 4 % faster with 4
// than with 3, 2 % faster again with 5, slower with 6)
__global__ void __launch_bounds__(32 * kBatchMaxLines, std::is_same<Pol, F32>::value ? 5 : 2)
    k_batch_queue(const __grid_constant__ QueueArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ QueueItem it;
    if (threadIdx.x == 0) {
        int p = 0, i = 0, t = 0;
        it.go = take_item(a, &p, &i, &t) ? 1 : 0;
        it.pass = p;
        it.inst = i;
        it.tile = t;
    }
    __syncthreads();
    if (!it.go) return;
    queue_pass<Pol, D, 0>(a, it, smem_raw);
    queue_pass<Pol, D, 1>(a, it, smem_raw);
    queue_pass<Pol, D, 2>(a, it, smem_raw);
    if constexpr (D == 3) {
        queue_pass<Pol, D, 3>(a, it, smem_raw);
        queue_pass<Pol, D, 4>(a, it, smem_raw);
    }
}

// ------------------------------------------------------------------ tables
// Constants of the FMA-form stages (slot-major blocks, see gindex in gsm_fft.cuh),
// one thread per (stage, j).  For stage radix R with Ns, forward twiddle
// W_t = exp(-2 pi i q / D), q = j t, D = R Ns: with K = round(4 q / D) and
// m = q - K D/4 (|m| <= D/8), W_t = i^(-K) exp(-2 pi i m / D), so k_t = -K mod 4,
// f_t = cos(2 pi m / D), tau_t = -tan(2 pi m / D).
struct GStage {
    int R;
    long Ns, off;   // off: first double of the stage's constants
};
struct GTableDesc {
    int n;
    GStage s[kMaxStages];
};

__global__ void k_gtable(GTableDesc d, double *out)
{
    const long idx = blockIdx.x * (long)blockDim.x + threadIdx.x;
    long base = 0;
    int st = 0;
    for (; st < d.n && idx >= base + d.s[st].Ns; ++st) base += d.s[st].Ns;
    if (st >= d.n) return;
    const int R = d.s[st].R;
    const long Ns = d.s[st].Ns, j = idx - base, D = R * Ns;
    double f[8], tau[8];
    int codes = 0;
    f[0] = 1.0;
    tau[0] = 0.0;
    for (int t = 1; t < R; ++t) {
        const long q = j * t;
        const long K = (4 * q + D / 2) / D;
        const long m = q - K * (D / 4);
        const int k = (int)((4 - (K & 3)) & 3);
        double sn, cs;
        sincospi(2.0 * (double)m / (double)D, &sn, &cs);
        f[t] = cs;
        tau[t] = (k & 1) ? sn / cs : -sn / cs;   // tau sigma_t, sigma_t = -1 for odd k
        codes |= k << (2 * (t - 1));
    }
    double *cj = out + d.s[st].off + gindex(R, j);
    auto c = [&](int q) -> double & { return cj[q * kGBlk]; };
    if (R == 8) {
        for (int t = 1; t < 8; ++t) c(t - 1) = tau[t];
        for (int t = 0; t < 4; ++t) c(7 + t) = f[t + 4] / f[t];
        c(11) = f[2];
        c(12) = f[3] / f[1];
        c(13) = f[1];
        c(14) = f[1] * 0.707106781186547524400844362104849039;
        c(15) = __hiloint2double(0, codes);
    } else if (R == 4) {
        for (int t = 1; t < 4; ++t) c(t - 1) = tau[t];
        c(3) = f[2];
        c(4) = f[3] / f[1];
        c(5) = f[1];
        c(6) = __hiloint2double(0, codes);
        c(7) = 0.0;
    } else {
        c(0) = tau[1];
        c(1) = f[1];
        c(2) = __hiloint2double(0, codes);
        c(3) = 0.0;
    }
}

// Fills the FMA-form constants of schedule sc at `dst` (just after the M
// twiddles of an FP64 table, so 16-byte aligned).
void launch_g8table(const Sched &sc, double2 *dst, cudaStream_t st)
{
    GTableDesc d;
    d.n = 0;
    long Ns = 1, entries = 0;
    for (int i = 0; i < sc.nst; ++i) {
        if (gtabled_at(sc.r[i], Ns)) {
            d.s[d.n].R = sc.r[i];
            d.s[d.n].Ns = Ns;
            d.s[d.n].off = (long)gtable_offset(sc, i);
            ++d.n;
            entries += Ns;
        }
        Ns *= sc.r[i];
    }
    if (entries > 0) k_gtable<<<(entries + 127) / 128, 128, 0, st>>>(d, reinterpret_cast<double *>(dst));
}

// w[m] = exp(-2 pi i m / M) from sincospi in FP64, then rounded or split.
__global__ void k_twiddles(int M, int prec, void *out)
{
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    double sn, cs;
    sincospi(2.0 * m / M, &sn, &cs);
    const double re = cs, im = -sn;
    if (prec == GSM_FP64) {
        reinterpret_cast<double2 *>(out)[m] = make_double2(re, im);
    } else if (prec == GSM_FP32) {
        reinterpret_cast<float2 *>(out)[m] = make_float2((float)re, (float)im);
    } else {
        const df a = df_from_double(re), b = df_from_double(im);
        reinterpret_cast<float4 *>(out)[m] = make_float4(a.hi, a.lo, b.hi, b.lo);
    }
}

__global__ void k_mult_convert(const double *in, size_t count, int prec, void *out)
{
    const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i >= count) return;
    if (prec == GSM_FP32) {
        reinterpret_cast<float *>(out)[i] = (float)in[i];
    } else {
        const df a = df_from_double(in[i]);
        reinterpret_cast<float2 *>(out)[i] = make_float2(a.hi, a.lo);
    }
}

// ------------------------------------------------------------------ Hartree energy
template <class T>
__global__ void k_psi_to_rho(const T *__restrict__ psi, T *__restrict__ rho, size_t N)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
        const T a = psi[2 * i], b = psi[2 * i + 1];
        rho[i] = a * a + b * b;
    }
}

// partial[block] = sum |psi|^2 u ; grad = 2 h^3 u psi
template <class T>
__global__ void k_energy_grad(const T *__restrict__ psi, const T *__restrict__ u, T *__restrict__ grad,
                              double cell, size_t N, double *partial)
{
    __shared__ double red[256];
    double acc = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
        const double a = psi[2 * i], b = psi[2 * i + 1], v = u[i];
        acc += (a * a + b * b) * v;
        if (grad) {
            grad[2 * i] = (T)(2.0 * cell * v * a);
            grad[2 * i + 1] = (T)(2.0 * cell * v * b);
        }
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
        if (threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

template <class T>
__global__ void k_energy_final(const double *partial, int nparts, double cell, T *energy)
{
    __shared__ double red[256];
    double acc = 0.0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) acc += partial[i];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
        if (threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
        __syncthreads();
    }
    if (threadIdx.x == 0) *energy = (T)(0.5 * cell * red[0]);
}

constexpr int kEnergyBlocks = 1024;

// ------------------------------------------------------------------ launching
// The dynamic shared-memory limit is per kernel function, shared by every
// plan; it is always raised to the device's opt-in maximum (never lowered) so
// that one plan cannot shrink the limit another plan launches with.
template <class K>
cudaError_t raise_smem(K kernel, size_t smem)
{
    if (smem <= 48 * 1024) return cudaSuccess;
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    if ((size_t)optin < smem) return cudaErrorInvalidValue;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
}

template <class Pol>
size_t pass_smem(int M, int nl) { return (size_t)nl * line_stride<Pol>(M) * sizeof(S_t<Pol>); }

// Launch shape for lines of length M: emax elements per thread (8 or 16),
// gthr = threads per line (a multiple of 32 with gthr * emax >= M), nl lines
// (groups) per CTA, nthr = nl * gthr <= kMaxThreads.  Groups larger than a
// warp in a CTA of several groups use named barriers 1..nl (nl <= 15).
inline int round32(int x) { return ((x + 31) / 32) * 32; }

template <class Pol>
bool make_cfg(int M, int nl, int emax, PassCfg *c, int maxt = kMaxThreads)
{
    const int gthr = std::max(32, round32((M + emax - 1) / emax));
    if (gthr > maxt || nl < 1 || nl * gthr > maxt) return false;
    if (gthr > 32 && nl > 1 && nl > 15) return false;
    if (pass_smem<Pol>(M, nl) > 200 * 1024) return false;
    c->nl = nl;
    c->gthr = gthr;
    c->nthr = nl * gthr;
    c->emax = emax;
    c->smem = pass_smem<Pol>(M, nl);
    return true;
}

// Default shape before any tuning: 8 elements per thread when a line fits
// 512 threads that way, else 16; as many lines as requested that fit.
template <class Pol>
PassCfg choose_cfg(int M, int nl_want, bool conv = false)
{
    PassCfg c;
    const int emax = (M <= 8 * kMaxThreads) ? 8 : 16;
    const int maxt = conv ? conv_max_threads<Pol>(emax) : xy_max_threads<Pol>(emax);
    for (int nl = std::max(1, nl_want); nl >= 1; nl /= 2)
        if (make_cfg<Pol>(M, nl, emax, &c, maxt)) return c;
    make_cfg<Pol>(M, 1, 16, &c);
    return c;
}

// Calls f(std::integral_constant<int, E>) with E = c.emax.
template <class F>
void with_emax(const PassCfg &c, F &&f)
{
    if (c.emax == 8) f(std::integral_constant<int, 8>());
    else f(std::integral_constant<int, 16>());
}

template <class Pol>
gsm_status_t configure_t(Plan *p)
{
    const int cw = (int)(128 / sizeof(S_t<Pol>));   // complex values per 128 bytes
    const int d = p->d;
    p->cfg_xf = choose_cfg<Pol>(p->M[0], std::max(1, cw / 2));
    p->cfg_xi = p->cfg_xf;
    if (d == 3) {
        p->cfg_yf = choose_cfg<Pol>(p->M[1], cw);
        p->cfg_yi = p->cfg_yf;
        p->cfg_conv = choose_cfg<Pol>(p->M[2], std::max(1, 4096 / p->M[2]), true);
    } else {
        p->cfg_conv = choose_cfg<Pol>(p->M[1], std::max(1, 4096 / p->M[1]), true);
        // long lines: two half-length transforms per line on a cluster of two CTAs
        // (options.debug bit 1 keeps one CTA per line, for comparisons)
        p->split_conv = p->M[1] >= kSplitMinM && (p->opt.debug & 2) == 0;
        if (p->split_conv) {
            if (!make_cfg<Pol>(p->M[1] / 2, 1, 16, &p->cfg_split) || p->cfg_split.nthr > kSplitThreads) {
                set_error("no launch shape for the split conv pass");
                return GSM_ERR_UNSUPPORTED_SIZE;
            }
            GSM_CUDA_TRY(raise_smem(k_conv_split<Pol, 16>, p->cfg_split.smem));
        }
        // the same for the x forward pass
        p->split_x = p->M[0] >= kSplitMinM && p->M[0] == 2 * p->n[0] && (p->opt.debug & 2) == 0;
        if (p->split_x) {
            if (!make_cfg<Pol>(p->M[0] / 2, 1, 16, &p->cfg_xsplit) || p->cfg_xsplit.nthr > kSplitThreads) {
                set_error("no launch shape for the split x pass");
                return GSM_ERR_UNSUPPORTED_SIZE;
            }
            GSM_CUDA_TRY(raise_smem(k_xf_split<Pol, 16>, p->cfg_xsplit.smem));
        }
    }
    cudaError_t e = cudaSuccess;
    auto chk = [&](cudaError_t x) { if (e == cudaSuccess) e = x; };
    with_emax(p->cfg_xf, [&](auto E) { chk(raise_smem(k_xf<Pol, E()>, p->cfg_xf.smem)); });
    with_emax(p->cfg_xi, [&](auto E) { chk(raise_smem(k_xi<Pol, E()>, p->cfg_xi.smem)); });
    with_emax(p->cfg_conv, [&](auto E) { chk(raise_smem(k_conv<Pol, E()>, p->cfg_conv.smem)); });
    if (d == 3) {
        with_emax(p->cfg_yf, [&](auto E) { chk(raise_smem(k_yf<Pol, E()>, p->cfg_yf.smem)); });
        with_emax(p->cfg_yi, [&](auto E) { chk(raise_smem(k_yi<Pol, E()>, p->cfg_yi.smem)); });
    }
    GSM_CUDA_TRY(e);
    // workspace
    const size_t cb = sizeof(S_t<Pol>);
    const size_t hx = p->n[0] + 1;
    if (d == 3) {
        p->work1_bytes = cb * (size_t)p->n[2] * hx * p->n[1];
        p->work2_bytes = cb * hx * (size_t)p->M[1] * p->n[2];
    } else {
        p->work1_bytes = cb * hx * p->n[1];
        p->work2_bytes = 0;
    }
    GSM_CUDA_TRY(dev_alloc(&p->d_work1, p->work1_bytes));
    if (p->work2_bytes) GSM_CUDA_TRY(dev_alloc(&p->d_work2, p->work2_bytes));
    return GSM_OK;
}

// One pass of the apply: 3D passes 0..4 = xf, yf, conv, yi, xi; 2D 0..2 = xf, conv, xi.
template <class Pol>
void launch_pass_t(const Plan *p, int pass, const void *rho_v, void *u_v, cudaStream_t st)
{
    using io = typename Pol::io_t;
    using tw = typename Pol::tw_t;
    const io *rho = static_cast<const io *>(rho_v);
    io *u = static_cast<io *>(u_v);
    const int nx = p->n[0], ny = p->n[1], nz = p->d == 3 ? p->n[2] : 1;
    const int hx = nx + 1;
    S_t<Pol> *W1 = static_cast<S_t<Pol> *>(p->d_work1);
    S_t<Pol> *W2 = static_cast<S_t<Pol> *>(p->d_work2);
    const auto *mult = static_cast<const typename Pol::mult_t *>(p->d_mult);
    const tw *twx = static_cast<const tw *>(p->d_tw[0]);
    const tw *twy = static_cast<const tw *>(p->d_tw[1]);
    const tw *twxi = static_cast<const tw *>(p->d_twi[0]);
    const tw *twyi = static_cast<const tw *>(p->d_twi[1]);
    const int last = p->d == 3 ? 4 : 2;
    if constexpr (std::is_same<Pol, F32>::value) {
        if ((pass == 0 || pass == last) && p->M[0] == 512 && p->rr_conv) {
            if (pass == 0) launch_x_rr512_f32(false, rho, W1, ny, nz, twx, st);
            else launch_x_rr512_f32(true, W1, u, ny, nz, twx, st);
            return;
        }
    }
    if (pass == 0 && p->split_x) {
        const PassCfg &c = p->cfg_xsplit;
        const tw *twh = static_cast<const tw *>(p->d_twxh);
        k_xf_split<Pol, 16><<<2 * ((ny + 1) / 2), c.nthr, c.smem, st>>>(rho, W1, nx, ny, hx, p->sched_xh, twh, twx);
        return;
    }
    if (pass == 0) {
        const PassCfg &c = p->cfg_xf;
        dim3 g((ny + 2 * c.nl - 1) / (2 * c.nl), nz);
        with_emax(c, [&](auto E) {
            k_xf<Pol, E()><<<g, c.nthr, c.smem, st>>>(rho, W1, nx, ny, hx, p->sched_f[0], c.nl, c.gthr, twx);
        });
    } else if (pass == last) {
        const PassCfg &c = p->cfg_xi;
        dim3 g((ny + 2 * c.nl - 1) / (2 * c.nl), nz);
        with_emax(c, [&](auto E) {
            k_xi<Pol, E()><<<g, c.nthr, c.smem, st>>>(W1, u, nx, ny, hx, p->sched_i[0], c.nl, c.gthr, twxi);
        });
    } else if (p->d == 2) {
        const PassCfg &c = p->cfg_conv;
        if constexpr (std::is_same<Pol, F32>::value) {
            if (p->M[1] == 512 && p->rr_conv) {
                launch_conv_rr512_f32(W1, mult, hx, 0, 1, ny + 1, p->mult_full, twy, st);
                return;
            }
        }
        if (p->split_conv) {
            const PassCfg &cs = p->cfg_split;
            k_conv_split<Pol, 16><<<2 * hx, cs.nthr, cs.smem, st>>>(
                W1, mult, hx, ny + 1, p->sched_hf, p->sched_hi, static_cast<const tw *>(p->d_twh),
                static_cast<const tw *>(p->d_twhi), twy, p->mult_full ? 1 : 0);
            return;
        }
        with_emax(c, [&](auto E) {
            k_conv<Pol, E()><<<(hx + c.nl - 1) / c.nl, c.nthr, c.smem, st>>>(
                W1, mult, hx, ny, 0, 1, ny + 1, p->sched_f[1], p->sched_i[1], c.nl, c.gthr, twy, twyi,
                p->mult_full ? 1 : 0);
        });
    } else {
        const tw *twz = static_cast<const tw *>(p->d_tw[2]);
        const tw *twzi = static_cast<const tw *>(p->d_twi[2]);
        const int My = p->M[1];
        if (pass == 1) {
            if constexpr (std::is_same<Pol, F32>::value) {
                if (p->M[1] == 512 && p->rr_conv) {
                    launch_y_rr512_f32(false, W1, W2, nz, hx, twy, st);
                    return;
                }
            }
            const PassCfg &c = p->cfg_yf;
            dim3 g((nz + c.nl - 1) / c.nl, hx);
            with_emax(c, [&](auto E) {
                k_yf<Pol, E()><<<g, c.nthr, c.smem, st>>>(W1, W2, ny, nz, hx, p->sched_f[1], c.nl, c.gthr, twy);
            });
        } else if (pass == 2) {
            const PassCfg &c = p->cfg_conv;
            const int nlines = hx * My;
            if constexpr (std::is_same<Pol, F32>::value) {
                if (p->M[2] == 512 && p->rr_conv) {
                    launch_conv_rr512_f32(W2, mult, nlines, 1, My, ny + 1, p->mult_full, twz, st);
                    return;
                }
            }
            with_emax(c, [&](auto E) {
                k_conv<Pol, E()><<<(nlines + c.nl - 1) / c.nl, c.nthr, c.smem, st>>>(
                    W2, mult, nlines, nz, 1, My, ny + 1, p->sched_f[2], p->sched_i[2], c.nl, c.gthr, twz, twzi,
                    p->mult_full ? 1 : 0);
            });
        } else {
            if constexpr (std::is_same<Pol, F32>::value) {
                if (p->M[1] == 512 && p->rr_conv) {
                    launch_y_rr512_f32(true, W2, W1, nz, hx, twy, st);
                    return;
                }
            }
            const PassCfg &c = p->cfg_yi;
            dim3 g((nz + c.nl - 1) / c.nl, hx);
            with_emax(c, [&](auto E) {
                k_yi<Pol, E()><<<g, c.nthr, c.smem, st>>>(W2, W1, ny, nz, hx, p->sched_i[1], c.nl, c.gthr, twyi);
            });
        }
    }
}

template <class Pol>
gsm_status_t apply_t(const Plan *p, const void *rho, void *u, cudaStream_t st)
{
    const int np = p->d == 3 ? 5 : 3;
    for (int pass = 0; pass < np; ++pass) launch_pass_t<Pol>(p, pass, rho, u, st);
    GSM_CUDA_TRY(cudaGetLastError());
    return GSM_OK;
}

template <class Pol>
gsm_status_t pass_t(const Plan *p, int pass, const void *rho, void *u, cudaStream_t st)
{
    launch_pass_t<Pol>(p, pass, rho, u, st);
    GSM_CUDA_TRY(cudaGetLastError());
    return GSM_OK;
}

// ------------------------------------------------------------------ autotuning
// Each pass has its own launch shape; the tuner times candidate shapes of
// one pass at a time (the others keep theirs) and keeps the fastest.
template <class Pol>
cudaError_t raise_pass_smem(const Plan *p, int pass, const PassCfg &c)
{
    const int last = p->d == 3 ? 4 : 2;
    cudaError_t e = cudaSuccess;
    with_emax(c, [&](auto E) {
        if (pass == 0) e = raise_smem(k_xf<Pol, E()>, c.smem);
        else if (pass == last) e = raise_smem(k_xi<Pol, E()>, c.smem);
        else if (p->d == 2 || pass == 2) e = raise_smem(k_conv<Pol, E()>, c.smem);
        else if (pass == 1) e = raise_smem(k_yf<Pol, E()>, c.smem);
        else e = raise_smem(k_yi<Pol, E()>, c.smem);
    });
    return e;
}

PassCfg *pass_cfg(Plan *p, int pass)
{
    if (p->d == 3) {
        PassCfg *c[5] = {&p->cfg_xf, &p->cfg_yf, &p->cfg_conv, &p->cfg_yi, &p->cfg_xi};
        return c[pass];
    }
    PassCfg *c[3] = {&p->cfg_xf, &p->cfg_conv, &p->cfg_xi};
    return c[pass];
}

int pass_len(const Plan *p, int pass)
{
    if (p->d == 3) {
        const int m[5] = {p->M[0], p->M[1], p->M[2], p->M[1], p->M[0]};
        return m[pass];
    }
    const int m[3] = {p->M[0], p->M[1], p->M[0]};
    return m[pass];
}

std::mutex g_tune_mutex;

bool same_sched(const Sched &a, const Sched &b)
{
    if (a.M != b.M || a.nst != b.nst) return false;
    for (int i = 0; i < a.nst; ++i)
        if (a.r[i] != b.r[i]) return false;
    return true;
}

std::string tune_key(const Plan *p, int pass)
{
    cudaDeviceProp prop;
    int dev = 0;
    cudaGetDevice(&dev);
    std::string name = "gpu";
    if (cudaGetDeviceProperties(&prop, dev) == cudaSuccess) name = prop.name;
    for (char &ch : name)
        if (ch == ' ') ch = '_';
    char buf[256];
    snprintf(buf, sizeof(buf), "v4 %s p%d d%d n%d,%d,%d pass%d", name.c_str(), (int)p->opt.precision, p->d, p->n[0],
             p->n[1], p->d == 3 ? p->n[2] : 1, pass);
    return buf;
}

std::string sched_str(const Sched &sc)
{
    std::string out;
    for (int i = 0; i < sc.nst; ++i) {
        if (i) out += '.';
        out += std::to_string((int)sc.r[i]);
    }
    return out;
}

bool sched_parse(const char *txt, int M, bool forward, Sched *sc)
{
    int r[kMaxStages], n = 0;
    const char *c = txt;
    while (*c && n < kMaxStages) {
        char *end = nullptr;
        const long v = strtol(c, &end, 10);
        if (end == c) break;
        r[n++] = (int)v;
        c = end;
        if (*c != '.') break;
        ++c;
    }
    return make_sched_order(M, r, n, forward, sc);
}

// The axis whose schedules pass `pass` uses, and which of them: 3D xf, yf
// the forward, xi, yi the inverse, conv both (axis z); 2D xf, xi and conv
// (both, axis y).
void pass_axis(const Plan *p, int pass, int *axis, bool *fwd, bool *inv)
{
    const int last = p->d == 3 ? 4 : 2;
    const int conv = p->d == 3 ? 2 : 1;
    *fwd = *inv = false;
    if (pass == 0) { *axis = 0; *fwd = true; }
    else if (pass == last) { *axis = 0; *inv = true; }
    else if (pass == conv) { *axis = p->d - 1; *fwd = *inv = true; }
    else if (pass == 1) { *axis = 1; *fwd = true; }
    else { *axis = 1; *inv = true; }
}

// FP32 passes with padded length 512 run register-resident kernels with a
// fixed decomposition: no schedule to choose.
bool pass_uses_rr(const Plan *p, int pass)
{
    int axis;
    bool f, i;
    pass_axis(p, pass, &axis, &f, &i);
    return p->opt.precision == GSM_FP32 && p->rr_conv && p->M[axis] == 512;
}

// The split 2D conv has a fixed launch shape and half-length schedules of its own.
// Largest CTA of a pass's kernel for a shape with emax elements per thread.
template <class Pol>
int pass_max_threads(const Plan *p, int pass, int emax)
{
    const bool conv = p->d == 3 ? pass == 2 : pass == 1;
    return conv ? conv_max_threads<Pol>(emax) : xy_max_threads<Pol>(emax);
}

bool pass_is_split(const Plan *p, int pass)
{
    return p->d == 2 && ((pass == 1 && p->split_conv) || (pass == 0 && p->split_x));
}

// Factorisations of M into radices 8, 4, 2, 5, 3 in the order fft_line runs
// them, with at most one stage more than the default schedule; the default
// first, at most `cap`.
void factorise(int M, int from_rank, std::vector<int> &cur, int max_st, std::vector<std::vector<int>> &out)
{
    static const int radices[5] = {8, 4, 2, 5, 3};
    if (M == 1) {
        out.push_back(cur);
        return;
    }
    if ((int)cur.size() >= max_st) return;
    for (int k = from_rank; k < 5; ++k)
        if (M % radices[k] == 0) {
            cur.push_back(radices[k]);
            factorise(M / radices[k], k, cur, max_st, out);
            cur.pop_back();
        }
}

std::vector<Sched> sched_factorisations(int M, size_t cap)
{
    Sched def;
    std::vector<Sched> out;
    if (!make_sched(M, &def)) return out;
    out.push_back(def);
    std::vector<std::vector<int>> all;
    std::vector<int> cur;
    factorise(M, 0, cur, def.nst + 1, all);
    std::sort(all.begin(), all.end(), [](const std::vector<int> &x, const std::vector<int> &y) {
        return x.size() < y.size();
    });
    for (const auto &f : all) {
        if (out.size() >= cap) break;
        Sched sc;
        if (!make_sched_order(M, f.data(), (int)f.size(), true, &sc)) continue;
        bool seen = false;
        for (const Sched &o : out) seen |= same_sched(o, sc);
        if (!seen) out.push_back(sc);
    }
    return out;
}

// The inverse schedule whose first stage fuses with the last stage of the
// forward f: f's last radix, then f's other radices in run order.
Sched fused_inverse(const Sched &f)
{
    Sched i = f;
    i.r[0] = f.r[f.nst - 1];
    for (int k = 0; k + 1 < f.nst; ++k) i.r[k + 1] = f.r[k];
    return i;
}

// Candidate (forward, inverse) schedules of pass `pass`, the current pair
// first: single-direction passes vary their own direction over the
// factorisations of M; the conv pass tries, for each factorisation, the
// inverse whose first stage fuses with the forward's last, and the same
// order both ways.
std::vector<std::pair<Sched, Sched>> sched_candidates(const Plan *p, int pass)
{
    int axis;
    bool f, i;
    pass_axis(p, pass, &axis, &f, &i);
    const int M = p->M[axis];
    std::vector<std::pair<Sched, Sched>> out;
    out.push_back({p->sched_f[axis], p->sched_i[axis]});
    auto add = [&](const Sched &a, const Sched &b) {
        if (!axis_pair_ok(p, axis, a, b)) return;
        for (const auto &o : out)
            if (same_sched(o.first, a) && same_sched(o.second, b)) return;
        out.push_back({a, b});
    };
    const std::vector<Sched> fz = sched_factorisations(M, 6);
    if (f && i) {
        for (const Sched &a : fz) {
            if (a.nst >= 2) add(a, fused_inverse(a));
            add(a, a);
        }
    } else if (f) {
        for (const Sched &a : fz) add(a, p->sched_i[axis]);
    } else {
        for (const Sched &b : fz) add(p->sched_f[axis], b);
    }
    return out;
}

gsm_status_t apply_axis_pair(Plan *p, int axis, const Sched &a, const Sched &b, cudaStream_t st)
{
    if (same_sched(p->sched_f[axis], a) && same_sched(p->sched_i[axis], b)) return GSM_OK;
    return set_axis_pair(p, axis, a, b, st);
}

bool cache_lookup(const char *path, const std::string &key, int *nl, int *emax, std::string *fs, std::string *is)
{
    FILE *f = fopen(path, "r");
    if (!f) return false;
    char line[512];
    bool hit = false;
    while (fgets(line, sizeof(line), f)) {
        const size_t kl = key.size();
        if (strncmp(line, key.c_str(), kl) == 0 && line[kl] == ' ') {
            int a = 0, b = 0;
            char sf[64] = {0}, si[64] = {0};
            if (sscanf(line + kl, " nl=%d emax=%d f=%63s i=%63s", &a, &b, sf, si) == 4) {
                *nl = a;
                *emax = b;
                *fs = sf;
                *is = si;
                hit = true;
            }
        }
    }
    fclose(f);
    return hit;
}

template <class Pol>
float time_pass(const Plan *p, int pass, const void *rho, void *u, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1,
                cudaError_t *err)
{
    launch_pass_t<Pol>(p, pass, rho, u, st);
    cudaEventRecord(e0, st);
    for (int r = 0; r < 3; ++r) launch_pass_t<Pol>(p, pass, rho, u, st);
    cudaEventRecord(e1, st);
    *err = cudaEventSynchronize(e1);
    if (*err == cudaSuccess) *err = cudaGetLastError();
    float ms = 0.f;
    if (*err == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
    return ms / 3.f;
}

template <class Pol>
gsm_status_t autotune_t(Plan *p, cudaStream_t st, std::string *report)
{
    using io = typename Pol::io_t;
    size_t N = 1;
    for (int a = 0; a < p->d; ++a) N *= (size_t)p->n[a];
    DevTemp rho_buf, u_buf;
    GSM_CUDA_TRY(dev_alloc(&rho_buf.p, N * sizeof(io)));
    GSM_CUDA_TRY(dev_alloc(&u_buf.p, N * sizeof(io)));
    void *rho = rho_buf.p, *u = u_buf.p;
    GSM_CUDA_TRY(cudaMemsetAsync(rho, 0, N * sizeof(io), st));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const char *cache = getenv("GSM_AUTOTUNE_CACHE");
    const int np = p->d == 3 ? 5 : 3;
    char buf[320];
    gsm_status_t s = GSM_OK;
    Sched keep_f[3], keep_i[3];   // put back if the tuning fails part-way
    for (int a = 0; a < p->d; ++a) {
        keep_f[a] = p->sched_f[a];
        keep_i[a] = p->sched_i[a];
    }
    if (e == cudaSuccess)
        for (int pass = 0; pass < np; ++pass) launch_pass_t<Pol>(p, pass, rho, u, st);
    for (int pass = 0; pass < np && e == cudaSuccess && s == GSM_OK; ++pass) {
        PassCfg *cfg = pass_cfg(p, pass);
        const int M = pass_len(p, pass);
        int axis;
        bool df, di;
        pass_axis(p, pass, &axis, &df, &di);
        const std::string key = tune_key(p, pass);
        int cnl = 0, cem = 0;
        std::string cf, ci;
        if (cache) {
            std::lock_guard<std::mutex> lock(g_tune_mutex);
            PassCfg c;
            Sched a, b;
            if (cache_lookup(cache, key, &cnl, &cem, &cf, &ci) && make_cfg<Pol>(M, cnl, cem, &c, pass_max_threads<Pol>(p, pass, cem)) &&
                sched_parse(cf.c_str(), p->M[axis], true, &a) && sched_parse(ci.c_str(), p->M[axis], false, &b) &&
                raise_pass_smem<Pol>(p, pass, c) == cudaSuccess) {
                s = apply_axis_pair(p, axis, df ? a : p->sched_f[axis], di ? b : p->sched_i[axis], st);
                if (s != GSM_OK) break;
                *cfg = c;
                snprintf(buf, sizeof(buf), "pass %d M=%d cached nl=%d gthr=%d emax=%d fwd=%s inv=%s\n", pass, M, c.nl,
                         c.gthr, c.emax, sched_str(p->sched_f[axis]).c_str(), sched_str(p->sched_i[axis]).c_str());
                *report += buf;
                continue;
            }
        }
        if (pass_is_split(p, pass)) {
            snprintf(buf, sizeof(buf), "pass %d M=%d split into two halves on a CTA pair (fixed shape)\n", pass, M);
            *report += buf;
            continue;
        }
        // 1. the radix schedule, with the current launch shape
        if (!pass_uses_rr(p, pass)) {
            const auto cands = sched_candidates(p, pass);
            size_t best_i = 0;
            float best_ms = 1e30f;
            for (size_t ci2 = 0; ci2 < cands.size() && e == cudaSuccess; ++ci2) {
                s = apply_axis_pair(p, axis, cands[ci2].first, cands[ci2].second, st);
                if (s != GSM_OK) break;
                const float ms = time_pass<Pol>(p, pass, rho, u, st, e0, e1, &e);
                if (e != cudaSuccess) break;
                snprintf(buf, sizeof(buf), "pass %d M=%d schedule fwd=%s inv=%s: %.4f ms\n", pass, M,
                         sched_str(cands[ci2].first).c_str(), sched_str(cands[ci2].second).c_str(), ms);
                *report += buf;
                if (ms < best_ms) {
                    best_ms = ms;
                    best_i = ci2;
                }
            }
            if (s != GSM_OK || e != cudaSuccess) break;
            s = apply_axis_pair(p, axis, cands[best_i].first, cands[best_i].second, st);
            if (s != GSM_OK) break;
        }
        // 2. the launch shape (elements per thread, lines per CTA) with that schedule
        PassCfg best = *cfg;
        float best_ms = 1e30f;
        const int nls[] = {1, 2, 3, 4, 6, 8, 12, 16};
        for (int emax : {8, 16}) {
            for (int nl : nls) {
                PassCfg c;
                if (!make_cfg<Pol>(M, nl, emax, &c, pass_max_threads<Pol>(p, pass, emax))) continue;
                if (raise_pass_smem<Pol>(p, pass, c) != cudaSuccess) continue;
                *cfg = c;
                const float ms = time_pass<Pol>(p, pass, rho, u, st, e0, e1, &e);
                if (e != cudaSuccess) break;
                snprintf(buf, sizeof(buf), "pass %d M=%d nl=%d gthr=%d emax=%d smem=%zu: %.4f ms\n", pass, M, c.nl,
                         c.gthr, c.emax, c.smem, ms);
                *report += buf;
                if (ms < best_ms) {
                    best_ms = ms;
                    best = c;
                }
            }
            if (e != cudaSuccess) break;
        }
        *cfg = best;
        if (cache && e == cudaSuccess) {
            std::lock_guard<std::mutex> lock(g_tune_mutex);
            FILE *f = fopen(cache, "a");
            if (f) {
                fprintf(f, "%s nl=%d emax=%d f=%s i=%s\n", key.c_str(), best.nl, best.emax,
                        sched_str(p->sched_f[axis]).c_str(), sched_str(p->sched_i[axis]).c_str());
                fclose(f);
            }
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s != GSM_OK || e != cudaSuccess) {
        const std::string msg = gsm_last_error();
        for (int a = 0; a < p->d; ++a) apply_axis_pair(p, a, keep_f[a], keep_i[a], st);
        set_error(msg);
    }
    if (s != GSM_OK) return s;
    GSM_CUDA_TRY(e);
    GSM_CUDA_TRY(cudaGetLastError());
    return GSM_OK;
}

template <class Pol>
gsm_status_t fft_hook_t(int M, int nlines, int sign, const double *in, double *out, cudaStream_t st)
{
    Sched sc;
    if (!make_sched(M, &sc)) {
        set_error("FFT length must be a product of 2, 3, 5 between 2 and 8192");
        return GSM_ERR_UNSUPPORTED_SIZE;
    }
    void *d_tw = nullptr;
    const size_t g8 = std::is_same<Pol, F64>::value ? g8_table_doubles(sc) : 0;
    GSM_CUDA_TRY(dev_alloc_async_bytes(&d_tw, sizeof(typename Pol::tw_t) * M + sizeof(double) * g8, st));
    k_twiddles<<<(M + 255) / 256, 256, 0, st>>>(M, Pol::kId, d_tw);
    if (g8 > 0) launch_g8table(sc, static_cast<double2 *>(d_tw) + M, st);
    const PassCfg c = choose_cfg<Pol>(M, std::max(1, 2048 / M));
    const auto *tw = static_cast<const typename Pol::tw_t *>(d_tw);
    const int blocks = (nlines + c.nl - 1) / c.nl;
    cudaError_t e = cudaSuccess;
    with_emax(c, [&](auto E) {
        if (sign < 0) {
            e = raise_smem(k_fft_hook<Pol, true, E()>, c.smem);
            if (e == cudaSuccess)
                k_fft_hook<Pol, true, E()><<<blocks, c.nthr, c.smem, st>>>((const double2 *)in, (double2 *)out,
                                                                           nlines, sc, c.nl, c.gthr, tw, 1);
        } else {
            e = raise_smem(k_fft_hook<Pol, false, E()>, c.smem);
            if (e == cudaSuccess)
                k_fft_hook<Pol, false, E()><<<blocks, c.nthr, c.smem, st>>>((const double2 *)in, (double2 *)out,
                                                                            nlines, sc, c.nl, c.gthr, tw, 1);
        }
    });
    if (e == cudaSuccess) e = cudaGetLastError();
    dev_free_async(d_tw, st);
    GSM_CUDA_TRY(e);
    return GSM_OK;
}

}  // namespace

// ------------------------------------------------------------------ exported
bool make_sched(int M, Sched *s)
{
    if (M < 2 || M > kMaxM) return false;
    s->M = M;
    s->nst = 0;
    int m = M;
    const int order[5] = {8, 4, 2, 5, 3};
    for (int r : order) {
        while (m % r == 0) {
            if (s->nst >= kMaxStages) return false;
            s->r[s->nst++] = r;
            m /= r;
        }
    }
    return m == 1;
}

size_t cplx_bytes(gsm_precision_t prec) { return prec == GSM_FP32 ? 8 : 16; }

namespace {

// Whether the table made for (M, schedule a) serves (M, schedule b): equal M
// and, in FP64 (whose tables end with the schedule's FMA-form constants),
// equal schedules.
bool table_serves(const Plan *p, const Sched &a, const Sched &b)
{
    return a.M == b.M && (p->opt.precision != GSM_FP64 || same_sched(a, b));
}

// The table of (axis, inverse?): an existing table that serves it, or a new one.
gsm_status_t table_for(Plan *p, int axis, bool inverse, cudaStream_t st, void **out)
{
    const Sched &want = inverse ? p->sched_i[axis] : p->sched_f[axis];
    for (int b = 0; b < p->d; ++b) {
        if (p->d_tw[b] && table_serves(p, p->sched_f[b], want) && !(b == axis && inverse == false)) {
            *out = p->d_tw[b];
            return GSM_OK;
        }
        if (p->d_twi[b] && table_serves(p, p->sched_i[b], want) && !(b == axis && inverse == true)) {
            *out = p->d_twi[b];
            return GSM_OK;
        }
    }
    const int M = want.M;
    const size_t g8 = p->opt.precision == GSM_FP64 ? g8_table_doubles(want) : 0;
    void *t = nullptr;
    GSM_CUDA_TRY(dev_alloc(&t, cplx_bytes(p->opt.precision) * M + sizeof(double) * g8));
    k_twiddles<<<(M + 255) / 256, 256, 0, st>>>(M, p->opt.precision, t);
    if (g8 > 0) launch_g8table(want, static_cast<double2 *>(t) + M, st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        dev_free(t);
        GSM_CUDA_TRY(e);
    }
    *out = t;
    return GSM_OK;
}

// Frees the table t unless a table slot of the plan still holds it.
void release_table(Plan *p, void *t)
{
    if (!t) return;
    for (int b = 0; b < 3; ++b)
        if (p->d_tw[b] == t || p->d_twi[b] == t) return;
    dev_free(t);
}

}  // namespace

gsm_status_t make_twiddles(Plan *p, int axis, cudaStream_t st)
{
    void *old_f = p->d_tw[axis], *old_i = p->d_twi[axis];
    p->d_tw[axis] = p->d_twi[axis] = nullptr;
    void *tf = nullptr, *ti = nullptr;
    gsm_status_t s = table_for(p, axis, false, st, &tf);
    if (s != GSM_OK) {
        p->d_tw[axis] = old_f;
        p->d_twi[axis] = old_i;
        return s;
    }
    p->d_tw[axis] = tf;
    s = table_for(p, axis, true, st, &ti);
    if (s != GSM_OK) {
        p->d_tw[axis] = old_f;
        p->d_twi[axis] = old_i;
        release_table(p, tf);
        return s;
    }
    p->d_twi[axis] = ti;
    // the device may still run work that reads the old tables: wait before freeing
    if ((old_f && old_f != tf && old_f != ti) || (old_i && old_i != tf && old_i != ti)) {
        GSM_CUDA_TRY(cudaStreamSynchronize(st));
        release_table(p, old_f);
        if (old_i != old_f) release_table(p, old_i);
    }
    return GSM_OK;
}

gsm_status_t make_xsplit_tables(Plan *p, cudaStream_t st)
{
    const int Mh = p->M[0] / 2;
    if (!make_sched(Mh, &p->sched_xh)) {
        set_error("half length of the split x pass is not a product of 2, 3 and 5");
        return GSM_ERR_UNSUPPORTED_SIZE;
    }
    const size_t g8 = p->opt.precision == GSM_FP64 ? g8_table_doubles(p->sched_xh) : 0;
    GSM_CUDA_TRY(dev_alloc(&p->d_twxh, cplx_bytes(p->opt.precision) * Mh + sizeof(double) * g8));
    k_twiddles<<<(Mh + 255) / 256, 256, 0, st>>>(Mh, p->opt.precision, p->d_twxh);
    if (g8 > 0) launch_g8table(p->sched_xh, static_cast<double2 *>(p->d_twxh) + Mh, st);
    GSM_CUDA_TRY(cudaGetLastError());
    return GSM_OK;
}

gsm_status_t make_split_tables(Plan *p, cudaStream_t st)
{
    const int Mh = p->M[1] / 2;
    if (!make_sched(Mh, &p->sched_hf)) {
        set_error("half length of the split conv is not a product of 2, 3 and 5");
        return GSM_ERR_UNSUPPORTED_SIZE;
    }
    // the inverse starts with the forward's last radix: fused with the multiplication
    p->sched_hi = p->sched_hf;
    p->sched_hi.r[0] = p->sched_hf.r[p->sched_hf.nst - 1];
    for (int k = 0; k + 1 < p->sched_hf.nst; ++k) p->sched_hi.r[k + 1] = p->sched_hf.r[k];
    const Sched *sc[2] = {&p->sched_hf, &p->sched_hi};
    void **dst[2] = {&p->d_twh, &p->d_twhi};
    for (int k = 0; k < 2; ++k) {
        const size_t g8 = p->opt.precision == GSM_FP64 ? g8_table_doubles(*sc[k]) : 0;
        if (k == 1 && g8 == 0) {   // without FMA-form constants one table serves both
            p->d_twhi = p->d_twh;
            break;
        }
        GSM_CUDA_TRY(dev_alloc(dst[k], cplx_bytes(p->opt.precision) * Mh + sizeof(double) * g8));
        k_twiddles<<<(Mh + 255) / 256, 256, 0, st>>>(Mh, p->opt.precision, *dst[k]);
        if (g8 > 0) launch_g8table(*sc[k], static_cast<double2 *>(*dst[k]) + Mh, st);
        GSM_CUDA_TRY(cudaGetLastError());
    }
    return GSM_OK;
}

bool make_sched_order(int M, const int *radices, int count, bool forward, Sched *s)
{
    if (M < 2 || M > kMaxM || count < 1 || count > kMaxStages || !radices) return false;
    long prod = 1;
    for (int i = 0; i < count; ++i) {
        const int r = radices[i];
        if (r != 8 && r != 4 && r != 2 && r != 5 && r != 3) return false;
        prod *= r;
    }
    if (prod != M) return false;
    if (forward && (radices[0] % 2) != 0) return false;   // the pruned first stage of the zero-padded transform
    s->M = M;
    s->nst = count;
    for (int i = 0; i < kMaxStages; ++i) s->r[i] = (unsigned char)(i < count ? radices[i] : 0);
    return true;
}

// Whether (forward f, inverse i) can run on axis `axis`: the forward and,
// except on the conv axis with a fused middle stage, the inverse in the order
// fft_line runs (8, 4, 2, 5, 3); on the conv axis the inverse may instead
// start with the forward's last radix, that stage being fused.
bool axis_pair_ok(const Plan *p, int axis, const Sched &f, const Sched &i)
{
    if (!sched_sorted_from(f, 0)) return false;
    if (sched_sorted_from(i, 0)) return true;
    return axis == p->d - 1 && fused_radix(f, i) != 0 && sched_sorted_from(i, 1);
}

gsm_status_t set_axis_pair(Plan *p, int axis, const Sched &f, const Sched &i, cudaStream_t st)
{
    if (axis < 0 || axis >= p->d || f.M != p->M[axis] || i.M != p->M[axis]) {
        set_error("schedule does not fit the axis");
        return GSM_ERR_INVALID_ARG;
    }
    if (!axis_pair_ok(p, axis, f, i)) {
        set_error("radices must run in the order 8, 4, 2, 5, 3; only the inverse of the conv axis may start "
                  "with the forward's last radix (fused with the multiplication)");
        return GSM_ERR_INVALID_ARG;
    }
    const Sched old_f = p->sched_f[axis], old_i = p->sched_i[axis];
    p->sched_f[axis] = f;
    p->sched_i[axis] = i;
    gsm_status_t s = make_twiddles(p, axis, st);
    if (s != GSM_OK) {
        p->sched_f[axis] = old_f;
        p->sched_i[axis] = old_i;
    }
    return s;
}

gsm_status_t set_axis_schedule(Plan *p, int axis, bool inverse, const Sched &sc, cudaStream_t st)
{
    if (axis < 0 || axis >= p->d) {
        set_error("axis out of range");
        return GSM_ERR_INVALID_ARG;
    }
    return set_axis_pair(p, axis, inverse ? p->sched_f[axis] : sc, inverse ? sc : p->sched_i[axis], st);
}

gsm_status_t make_pass_multiplier(Plan *p, cudaStream_t st)
{
    if (p->opt.precision == GSM_FP64) {
        p->d_mult = p->d_mult64;
        return GSM_OK;
    }
    const size_t eb = p->opt.precision == GSM_FP32 ? sizeof(float) : sizeof(float2);
    GSM_CUDA_TRY(dev_alloc(&p->d_mult, eb * p->mult_elems));
    k_mult_convert<<<(p->mult_elems + 255) / 256, 256, 0, st>>>(p->d_mult64, p->mult_elems, p->opt.precision,
                                                                  p->d_mult);
    GSM_CUDA_TRY(cudaGetLastError());
    return GSM_OK;
}

gsm_status_t configure_passes(Plan *p)
{
    for (int a = 0; a < p->d; ++a) {
        if (!make_sched(p->M[a], &p->sched_f[a])) {
            set_error("padded length 2n must be a product of 2, 3 and 5");
            return GSM_ERR_UNSUPPORTED_SIZE;
        }
        p->sched_i[a] = p->sched_f[a];
    }
    switch (p->opt.precision) {
    case GSM_FP64: return configure_t<F64>(p);
    case GSM_FP32: return configure_t<F32>(p);
    default: return configure_t<DF64>(p);
    }
}

gsm_status_t launch_apply(const Plan *p, const void *rho, void *u, cudaStream_t st)
{
    switch (p->opt.precision) {
    case GSM_FP64: return apply_t<F64>(p, rho, u, st);
    case GSM_FP32: return apply_t<F32>(p, rho, u, st);
    default: return apply_t<DF64>(p, rho, u, st);
    }
}

template <class Pol>
gsm_status_t x_slabs_t(const Plan *p, bool inverse, int z0, int z1, const void *rho_v, void *u_v,
                       cudaStream_t st)
{
    using io = typename Pol::io_t;
    using tw = typename Pol::tw_t;
    const int nx = p->n[0], ny = p->n[1], hx = nx + 1;
    const size_t in_off = (size_t)z0 * ny * nx, w_off = (size_t)z0 * hx * ny;
    S_t<Pol> *W1 = static_cast<S_t<Pol> *>(p->d_work1) + w_off;
    const tw *twx = static_cast<const tw *>(p->d_tw[0]);
    const tw *twxi = static_cast<const tw *>(p->d_twi[0]);
    if (z1 <= z0) return GSM_OK;
    if constexpr (std::is_same<Pol, F32>::value) {
        if (p->M[0] == 512 && p->rr_conv) {
            if (!inverse) launch_x_rr512_f32(false, static_cast<const io *>(rho_v) + in_off, W1, ny, z1 - z0, twx, st);
            else launch_x_rr512_f32(true, W1, static_cast<io *>(u_v) + in_off, ny, z1 - z0, twx, st);
            GSM_CUDA_TRY(cudaGetLastError());
            return GSM_OK;
        }
    }
    if (!inverse) {
        const PassCfg &c = p->cfg_xf;
        dim3 g((ny + 2 * c.nl - 1) / (2 * c.nl), z1 - z0);
        const io *rho = static_cast<const io *>(rho_v) + in_off;
        with_emax(c, [&](auto E) {
            k_xf<Pol, E()><<<g, c.nthr, c.smem, st>>>(rho, W1, nx, ny, hx, p->sched_f[0], c.nl, c.gthr, twx);
        });
    } else {
        const PassCfg &c = p->cfg_xi;
        dim3 g((ny + 2 * c.nl - 1) / (2 * c.nl), z1 - z0);
        io *u = static_cast<io *>(u_v) + in_off;
        with_emax(c, [&](auto E) {
            k_xi<Pol, E()><<<g, c.nthr, c.smem, st>>>(W1, u, nx, ny, hx, p->sched_i[0], c.nl, c.gthr, twxi);
        });
    }
    GSM_CUDA_TRY(cudaGetLastError());
    return GSM_OK;
}

gsm_status_t launch_x_slabs(const Plan *p, bool inverse, int z0, int z1, const void *rho, void *u, cudaStream_t st)
{
    if (p->d != 3 || z0 < 0 || z1 > p->n[2]) {
        set_error("x slabs: 3D plans and 0 <= z0 <= z1 <= nz only");
        return GSM_ERR_INVALID_ARG;
    }
    switch (p->opt.precision) {
    case GSM_FP64: return x_slabs_t<F64>(p, inverse, z0, z1, rho, u, st);
    case GSM_FP32: return x_slabs_t<F32>(p, inverse, z0, z1, rho, u, st);
    default: return x_slabs_t<DF64>(p, inverse, z0, z1, rho, u, st);
    }
}

gsm_status_t launch_pass(const Plan *p, int pass, const void *rho, void *u, cudaStream_t st)
{
    switch (p->opt.precision) {
    case GSM_FP64: return pass_t<F64>(p, pass, rho, u, st);
    case GSM_FP32: return pass_t<F32>(p, pass, rho, u, st);
    default: return pass_t<DF64>(p, pass, rho, u, st);
    }
}

template <class Pol>
gsm_status_t set_pass_shape_t(Plan *p, int pass, int nl, int emax)
{
    PassCfg c;
    if (!make_cfg<Pol>(pass_len(p, pass), nl, emax, &c, pass_max_threads<Pol>(p, pass, emax))) {
        set_error("launch shape not valid for this pass");
        return GSM_ERR_INVALID_ARG;
    }
    GSM_CUDA_TRY(raise_pass_smem<Pol>(p, pass, c));
    *pass_cfg(p, pass) = c;
    return GSM_OK;
}

gsm_status_t set_pass_shape(Plan *p, int pass, int nl, int emax)
{
    if (pass < 0 || pass >= (p->d == 3 ? 5 : 3)) {
        set_error("pass out of range");
        return GSM_ERR_INVALID_ARG;
    }
    switch (p->opt.precision) {
    case GSM_FP64: return set_pass_shape_t<F64>(p, pass, nl, emax);
    case GSM_FP32: return set_pass_shape_t<F32>(p, pass, nl, emax);
    default: return set_pass_shape_t<DF64>(p, pass, nl, emax);
    }
}

gsm_status_t autotune_plan(Plan *p, cudaStream_t st, std::string *report)
{
    switch (p->opt.precision) {
    case GSM_FP64: return autotune_t<F64>(p, st, report);
    case GSM_FP32: return autotune_t<F32>(p, st, report);
    default: return autotune_t<DF64>(p, st, report);
    }
}

gsm_status_t launch_fft_lines(int M, int nlines, int sign, gsm_precision_t prec, const double *in,
                              double *out, cudaStream_t st)
{
    switch (prec) {
    case GSM_FP64: return fft_hook_t<F64>(M, nlines, sign, in, out, st);
    case GSM_FP32: return fft_hook_t<F32>(M, nlines, sign, in, out, st);
    default: return fft_hook_t<DF64>(M, nlines, sign, in, out, st);
    }
}

template <class T>
static gsm_status_t hartree_t(Plan *p, const T *psi, T *u, T *energy, T *grad, cudaStream_t st)
{
    size_t N = 1;
    double cell = 1.0;
    for (int a = 0; a < p->d; ++a) {
        N *= (size_t)p->n[a];
        cell *= 2.0 * p->L * p->eta[a] / p->n[a];
    }
    if (!p->d_scratch) {
        GSM_CUDA_TRY(dev_alloc(&p->d_scratch, sizeof(double) * kEnergyBlocks));
        p->scratch_elems = kEnergyBlocks;
    }
    k_psi_to_rho<T><<<kEnergyBlocks, 256, 0, st>>>(psi, u, N);
    gsm_status_t s = launch_apply(p, u, u, st);
    if (s != GSM_OK) return s;
    k_energy_grad<T><<<kEnergyBlocks, 256, 0, st>>>(psi, u, grad, cell, N, p->d_scratch);
    k_energy_final<T><<<1, 256, 0, st>>>(p->d_scratch, kEnergyBlocks, cell, energy);
    GSM_CUDA_TRY(cudaGetLastError());
    return GSM_OK;
}

gsm_status_t launch_hartree(Plan *p, const void *psi, void *u, void *energy, void *grad, cudaStream_t st)
{
    if (p->opt.precision == GSM_FP32)
        return hartree_t<float>(p, (const float *)psi, (float *)u, (float *)energy, (float *)grad, st);
    return hartree_t<double>(p, (const double *)psi, (double *)u, (double *)energy, (double *)grad, st);
}

// ------------------------------------------------------------------ no-allocation FFT
// Scratch of gsm_fft_lines_noalloc: the tables of one transform length, the M
// twiddles (16-byte entries in FP64 and double-float, 8-byte in FP32) followed,
// in FP64, by the constants of the FMA-form stages, exactly as gsm_fft_lines
// builds them in its own allocation.  The largest need is M = 8192 in FP64,
// 131072 + 208896 = 339968 bytes.  A file-scope __device__ array, so every GPU
// that loads this library holds these 384 KiB until the process exits; every
// call shares it.
namespace {

constexpr size_t kStaticScratchBytes = 384 * 1024;
__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

typedef CUresult (*CtxGetCurrentFn)(CUcontext *);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long *);

// Identifier of the calling thread's current context (unique for the life of
// the process), or 0 if the driver does not give one.
unsigned long long current_context_id()
{
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<CtxGetCurrentFn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<CtxGetIdFn>(f);
        cudaGetLastError();
    });
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS)
        return 0;
    return id;
}

std::mutex g_static_mutex;
std::vector<std::pair<unsigned long long, void *>> g_static_addr;   // (context id, device address)

// The host-side name g_static_scratch is not a device address.  The device
// address is looked up with cudaGetSymbolAddress, with the caller's device
// current, once per context (device, or a new primary context after
// cudaDeviceReset), and remembered; while no context id is available (before
// the runtime has made one current) it is looked up on every call.
cudaError_t static_scratch_address(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long ctx = current_context_id();
    std::lock_guard<std::mutex> lock(g_static_mutex);
    if (ctx != 0)
        for (const auto &kv : g_static_addr)
            if (kv.first == ctx) {
                *out = kv.second;
                return cudaSuccess;
            }
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    if (ctx != 0) g_static_addr.emplace_back(ctx, p);
    *out = p;
    return cudaSuccess;
}

template <class Pol>
gsm_status_t fft_hook_static_t(int M, int nlines, int sign, const double *in, double *out, cudaStream_t st)
{
    Sched sc;
    if (!make_sched(M, &sc)) {
        set_error("FFT length must be a product of 2, 3, 5 between 2 and 8192");
        return GSM_ERR_UNSUPPORTED_SIZE;
    }
    const size_t g8 = std::is_same<Pol, F64>::value ? g8_table_doubles(sc) : 0;
    const size_t need = sizeof(typename Pol::tw_t) * (size_t)M + sizeof(double) * g8;
    if (need > kStaticScratchBytes) {
        set_error("FFT tables exceed the 384 KiB static scratch (M <= 8192)");
        return GSM_ERR_UNSUPPORTED_SIZE;
    }
    void *d_tw = nullptr;
    GSM_CUDA_TRY(static_scratch_address(&d_tw));
    // the same tables gsm_fft_lines builds, so the same arithmetic and the same
    // bits; every entry the FFT reads is written here first: nothing needs clearing
    k_twiddles<<<(M + 255) / 256, 256, 0, st>>>(M, Pol::kId, d_tw);
    if (g8 > 0) launch_g8table(sc, static_cast<double2 *>(d_tw) + M, st);
    const PassCfg c = choose_cfg<Pol>(M, std::max(1, 2048 / M));
    const auto *tw = static_cast<const typename Pol::tw_t *>(d_tw);
    const int blocks = (nlines + c.nl - 1) / c.nl;
    cudaError_t e = cudaSuccess;
    with_emax(c, [&](auto E) {
        if (sign < 0) {
            e = raise_smem(k_fft_hook<Pol, true, E()>, c.smem);
            if (e == cudaSuccess)
                k_fft_hook<Pol, true, E()><<<blocks, c.nthr, c.smem, st>>>((const double2 *)in, (double2 *)out,
                                                                           nlines, sc, c.nl, c.gthr, tw, 1);
        } else {
            e = raise_smem(k_fft_hook<Pol, false, E()>, c.smem);
            if (e == cudaSuccess)
                k_fft_hook<Pol, false, E()><<<blocks, c.nthr, c.smem, st>>>((const double2 *)in, (double2 *)out,
                                                                            nlines, sc, c.nl, c.gthr, tw, 1);
        }
    });
    GSM_CUDA_TRY(e);
    GSM_CUDA_TRY(cudaGetLastError());
    return GSM_OK;
}

}  // namespace

gsm_status_t launch_fft_lines_noalloc(int M, int nlines, int sign, gsm_precision_t prec, const double *in,
                                      double *out, cudaStream_t st)
{
    switch (prec) {
    case GSM_FP64: return fft_hook_static_t<F64>(M, nlines, sign, in, out, st);
    case GSM_FP32: return fft_hook_static_t<F32>(M, nlines, sign, in, out, st);
    default: return fft_hook_static_t<DF64>(M, nlines, sign, in, out, st);
    }
}


// ------------------------------------------------------------------ grouped batch, host side
namespace {

bool batch_eligible(const Plan *p)
{
    for (int a = 0; a < p->d; ++a) {
        if (p->M[a] > kBatchMaxM) return false;
        // FP32 plans that use the register-resident kernels apply alone, so that
        // a batch gives the same bits as gsm_apply
        if (p->opt.precision == GSM_FP32 && p->rr_conv && p->M[a] == 512) return false;
    }
    return true;
}

// Tile grid of pass `pass` of plan p for lines-per-CTA nl: (gx, gy).
void pass_grid(const Plan *p, int pass, int nl, int *gx, int *gy)
{
    const int nx = p->n[0], ny = p->n[1], nz = p->d == 3 ? p->n[2] : 1, hx = nx + 1;
    const int last = p->d == 3 ? 4 : 2;
    if (pass == 0 || pass == last) {
        *gx = (ny + 2 * nl - 1) / (2 * nl);
        *gy = nz;
    } else if (p->d == 2) {
        *gx = (hx + nl - 1) / nl;
        *gy = 1;
    } else if (pass == 2) {
        *gx = (hx * p->M[1] + nl - 1) / nl;
        *gy = 1;
    } else {
        *gx = (nz + nl - 1) / nl;
        *gy = hx;
    }
}

std::atomic<unsigned long long> g_batch_wait_ns{kBatchWaitDefaultNs};
std::atomic<int> g_batch_hold{-1};

template <class Pol>
gsm_status_t launch_queue_t(QueueArgs &a, const std::vector<const Plan *> &plans, const void *const *rho,
                              void *const *u, cudaStream_t st, bool dry)
{
    const int np = a.d == 3 ? 5 : 3;
    a.npass = np;
    size_t smem = 0;
    for (size_t i = 0; i < plans.size(); ++i) {
        const Plan *p = plans[i];
        InstDesc &d = a.inst[i];
        d.rho = rho[i];
        d.u = u[i];
        d.W1 = p->d_work1;
        d.W2 = p->d_work2;
        d.mult = p->d_mult;
        d.full = p->mult_full ? 1 : 0;
        for (int ax = 0; ax < 3; ++ax) {
            d.n[ax] = ax < p->d ? p->n[ax] : 1;
            d.M[ax] = ax < p->d ? p->M[ax] : 1;
            d.tw[ax] = ax < p->d ? p->d_tw[ax] : nullptr;
            d.twi[ax] = ax < p->d ? p->d_twi[ax] : nullptr;
            if (ax < p->d) {
                d.sc[ax] = p->sched_f[ax];
                d.sci[ax] = p->sched_i[ax];
            }
            if (ax < p->d) smem = std::max(smem, pass_smem<Pol>(p->M[ax], a.nl));
        }
        for (int pass = 0; pass < np; ++pass) {
            int gx, gy;
            pass_grid(p, pass, a.nl, &gx, &gy);
            d.gx[pass] = gx;
        }
    }
    // the queue: pass-major, instances in order within a pass, tiles in order
    int item = 0;
    for (int pass = 0; pass < np; ++pass) {
        a.start[pass] = item;
        a.tiles[pass][0] = 0;
        for (int i = 0; i < a.count; ++i) {
            int gx, gy;
            pass_grid(plans[i], pass, a.nl, &gx, &gy);
            a.tiles[pass][i + 1] = a.tiles[pass][i] + gx * gy;
        }
        item += a.tiles[pass][a.count];
    }
    for (int pass = np; pass <= kBatchPasses; ++pass) a.start[pass] = item;
    a.total = item;
    auto kernel = a.d == 3 ? k_batch_queue<Pol, 3> : k_batch_queue<Pol, 2>;
    cudaError_t e = raise_smem(kernel, smem);
    if (e == cudaSuccess && !dry) {
        // one CTA per item
        kernel<<<std::max(1, a.total), a.nl * 32, smem, st>>>(a);
        e = cudaGetLastError();
    }
    GSM_CUDA_TRY(e);
    return GSM_OK;
}

}  // namespace

size_t batch_state_bytes(int count) { return sizeof(unsigned) * kStateWords * (size_t)std::max(count, 1); }

void set_batch_wait(unsigned long long wait_ns, int hold)
{
    g_batch_wait_ns.store(wait_ns == 0 ? kBatchWaitDefaultNs : wait_ns);
    g_batch_hold.store(hold < 0 ? -1 : hold);
}

// u[i] = U_i * rho[i]: plans with all padded lengths <= 512 are grouped by
// (precision, dimension) into queue launches (k_batch_queue) of up to
// kBatchMax instances; the others are applied one by one.  Group g keeps its queue
// state at state + g * kStateWords (batch_state_bytes(count) bytes in all,
// zeroed here first).  dry: only prepare the kernels (shared-memory limits),
// launch nothing.
gsm_status_t launch_batched(int count, const Plan *const *plans, const void *const *rho, void *const *u,
                            int nl, cudaStream_t st, bool dry, unsigned *state)
{
    if (!dry) GSM_CUDA_TRY(cudaMemsetAsync(state, 0, batch_state_bytes(count), st));
    std::vector<int> done(count, 0);
    int group = 0;
    for (int i = 0; i < count; ++i) {
        if (done[i]) continue;
        if (!batch_eligible(plans[i])) {
            gsm_status_t s = dry ? GSM_OK : launch_apply(plans[i], rho[i], u[i], st);
            if (s != GSM_OK) return s;
            done[i] = 1;
            continue;
        }
        std::vector<const Plan *> grp;
        std::vector<const void *> r;
        std::vector<void *> w;
        for (int j = i; j < count && (int)grp.size() < kBatchMax; ++j) {
            if (done[j] || !batch_eligible(plans[j])) continue;
            if (plans[j]->opt.precision != plans[i]->opt.precision || plans[j]->d != plans[i]->d) continue;
            grp.push_back(plans[j]);
            r.push_back(rho[j]);
            w.push_back(u[j]);
            done[j] = 1;
        }
        QueueArgs *a = new (std::nothrow) QueueArgs();
        if (!a) {
            set_error("host allocation failed");
            return GSM_ERR_OOM;
        }
        a->count = (int)grp.size();
        a->d = plans[i]->d;
        a->nl = nl;
        a->state = state + (size_t)group * kStateWords;
        a->wait_ns = g_batch_wait_ns.load();
        a->hold = g_batch_hold.load();
        ++group;
        gsm_status_t s;
        switch (plans[i]->opt.precision) {
        case GSM_FP64: s = launch_queue_t<F64>(*a, grp, r.data(), w.data(), st, dry); break;
        case GSM_FP32: s = launch_queue_t<F32>(*a, grp, r.data(), w.data(), st, dry); break;
        default: s = launch_queue_t<DF64>(*a, grp, r.data(), w.data(), st, dry); break;
        }
        delete a;
        if (s != GSM_OK) return s;
    }
    return GSM_OK;
}

// Status of the queue launches whose queue state is at `state`, read
// after everything queued on `st`: GSM_ERR_TIMEOUT if a bounded wait ran out.
gsm_status_t batch_status(const unsigned *state, int count, cudaStream_t st)
{
    std::vector<unsigned> h(batch_state_bytes(count) / sizeof(unsigned));
    GSM_CUDA_TRY(cudaMemcpyAsync(h.data(), state, batch_state_bytes(count), cudaMemcpyDeviceToHost, st));
    GSM_CUDA_TRY(cudaStreamSynchronize(st));
    for (size_t g = 0; g * kStateWords < h.size(); ++g)
        if (h[g * kStateWords + 1] != 0) {
            set_error("a bounded wait of the batch kernel ran out; this batch's outputs are not valid");
            return GSM_ERR_TIMEOUT;
        }
    return GSM_OK;
}

}  // namespace gsm
