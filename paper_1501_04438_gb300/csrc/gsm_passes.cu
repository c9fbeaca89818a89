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
#include <algorithm>
#include <mutex>
#include <type_traits>

#include "gsm_internal.h"

namespace gsm {

namespace {

constexpr int kMaxThreads = 512;   // CTA size cap: leaves 128 registers per thread

template <class Pol>
using S_t = typename Pol::scplx;

// ------------------------------------------------------------------ pass xf
template <class Pol, int EMAX>
__global__ void __launch_bounds__(kMaxThreads) k_xf(const typename Pol::io_t *__restrict__ rho,
                                             S_t<Pol> *__restrict__ W1, int nx, int ny, int hx,
                                             Sched sc, int nl, const typename Pol::tw_t *__restrict__ tw)
{
    using R = typename Pol::real;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    S_t<Pol> *s = reinterpret_cast<S_t<Pol> *>(smem_raw);
    const int M = sc.M, LS = line_stride<Pol>(M);
    const int z = blockIdx.y;
    const int y0 = blockIdx.x * 2 * nl;
    const typename Pol::io_t *slab = rho + (size_t)z * ny * nx;
    for (int i = threadIdx.x; i < nl * M; i += blockDim.x) {
        const int l = i / M, x = i - l * M;
        const int ya = y0 + 2 * l;
        R a = Pol::zero(), b = Pol::zero();
        if (x < nx) {
            if (ya < ny) a = Pol::from_io(slab[(size_t)ya * nx + x]);
            if (ya + 1 < ny) b = Pol::from_io(slab[(size_t)(ya + 1) * nx + x]);
        }
        s[l * LS + pidx<Pol>(x)] = Pol::st(cx<R>{a, b});
    }
    __syncthreads();
    fft_lines<Pol, true, EMAX>(s, LS, sc, nl, tw, threadIdx.x, blockDim.x);
    // Z = A + iB with A, B the transforms of the two real rows:
    // 2A[k] = Z[k] + conj Z[-k], 2B[k] = -i (Z[k] - conj Z[-k]); the factor 2
    // is removed by the multiplier.
    S_t<Pol> *out = W1 + (size_t)z * hx * ny;
    for (int i = threadIdx.x; i < hx * nl; i += blockDim.x) {
        const int k = i / nl, l = i - k * nl;
        const cx<R> zk = Pol::ld(s[l * LS + pidx<Pol>(k)]);
        const cx<R> zm = cconj(Pol::ld(s[l * LS + pidx<Pol>(k == 0 ? 0 : M - k)]));
        const int ya = y0 + 2 * l;
        if (ya < ny) out[(size_t)k * ny + ya] = Pol::st(cadd(zk, zm));
        if (ya + 1 < ny) out[(size_t)k * ny + ya + 1] = Pol::st(cmul_negi(csub(zk, zm)));
    }
}

// ------------------------------------------------------------------ pass yf
template <class Pol, int EMAX>
__global__ void __launch_bounds__(kMaxThreads) k_yf(const S_t<Pol> *__restrict__ W1, S_t<Pol> *__restrict__ W2,
                                             int ny, int nz, int hx, Sched sc, int nl,
                                             const typename Pol::tw_t *__restrict__ tw)
{
    using R = typename Pol::real;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    S_t<Pol> *s = reinterpret_cast<S_t<Pol> *>(smem_raw);
    const int M = sc.M, LS = line_stride<Pol>(M);
    const int kx = blockIdx.y;
    const int z0 = blockIdx.x * nl;
    for (int i = threadIdx.x; i < nl * M; i += blockDim.x) {
        const int l = i / M, y = i - l * M;
        const int z = z0 + l;
        S_t<Pol> v = Pol::st(cx<R>{Pol::zero(), Pol::zero()});
        if (y < ny && z < nz) v = W1[((size_t)z * hx + kx) * ny + y];
        s[l * LS + pidx<Pol>(y)] = v;
    }
    __syncthreads();
    fft_lines<Pol, true, EMAX>(s, LS, sc, nl, tw, threadIdx.x, blockDim.x);
    S_t<Pol> *out = W2 + (size_t)kx * M * nz;
    for (int i = threadIdx.x; i < M * nl; i += blockDim.x) {
        const int ky = i / nl, l = i - ky * nl;
        const int z = z0 + l;
        if (z < nz) out[(size_t)ky * nz + z] = s[l * LS + pidx<Pol>(ky)];
    }
}

// ------------------------------------------------------------------ pass conv
// Lines of length n (stored) padded to M: forward, multiply by the real
// multiplier mult[row + min(k, M - k)], inverse, keep the first n.
// 3D: line = kx * My + ky, row = (kx * (ny + 1) + min(ky, My - ky)) * (nz + 1).
// 2D: line = kx, row = kx * (ny + 1).
template <class Pol, int EMAX>
__global__ void __launch_bounds__(kMaxThreads) k_conv(S_t<Pol> *__restrict__ W, const typename Pol::mult_t *__restrict__ mult,
                                               int nlines, int n, int is3d, int My, int ny1, Sched sc,
                                               int nl, const typename Pol::tw_t *__restrict__ tw)
{
    using R = typename Pol::real;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    S_t<Pol> *s = reinterpret_cast<S_t<Pol> *>(smem_raw);
    const int M = sc.M, LS = line_stride<Pol>(M);
    const int line0 = blockIdx.x * nl;
    for (int i = threadIdx.x; i < nl * M; i += blockDim.x) {
        const int l = i / M, z = i - l * M;
        const int line = line0 + l;
        S_t<Pol> v = Pol::st(cx<R>{Pol::zero(), Pol::zero()});
        if (z < n && line < nlines) v = W[(size_t)line * n + z];
        s[l * LS + pidx<Pol>(z)] = v;
    }
    __syncthreads();
    fft_lines<Pol, true, EMAX>(s, LS, sc, nl, tw, threadIdx.x, blockDim.x);
    const int h = n + 1;
    for (int i = threadIdx.x; i < nl * M; i += blockDim.x) {
        const int l = i / M, k = i - l * M;
        const int line = line0 + l;
        if (line >= nlines) continue;
        size_t row;
        if (is3d) {
            const int kx = line / My, ky = line - kx * My;
            const int fky = min(ky, My - ky);
            row = ((size_t)kx * ny1 + fky) * h;
        } else {
            row = (size_t)line * h;
        }
        const int fk = min(k, M - k);
        const R m = Pol::mult(mult[row + fk]);
        const int p = l * LS + pidx<Pol>(k);
        s[p] = Pol::st(cscale(Pol::ld(s[p]), m));
    }
    __syncthreads();
    fft_lines<Pol, false, EMAX>(s, LS, sc, nl, tw, threadIdx.x, blockDim.x);
    for (int i = threadIdx.x; i < nl * n; i += blockDim.x) {
        const int l = i / n, z = i - l * n;
        const int line = line0 + l;
        if (line < nlines) W[(size_t)line * n + z] = s[l * LS + pidx<Pol>(z)];
    }
}

// ------------------------------------------------------------------ pass yi
template <class Pol, int EMAX>
__global__ void __launch_bounds__(kMaxThreads) k_yi(const S_t<Pol> *__restrict__ W2, S_t<Pol> *__restrict__ W1,
                                             int ny, int nz, int hx, Sched sc, int nl,
                                             const typename Pol::tw_t *__restrict__ tw)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    S_t<Pol> *s = reinterpret_cast<S_t<Pol> *>(smem_raw);
    const int M = sc.M, LS = line_stride<Pol>(M);
    const int kx = blockIdx.y;
    const int z0 = blockIdx.x * nl;
    const S_t<Pol> *in = W2 + (size_t)kx * M * nz;
    for (int i = threadIdx.x; i < M * nl; i += blockDim.x) {
        const int ky = i / nl, l = i - ky * nl;
        const int z = z0 + l;
        if (z < nz) s[l * LS + pidx<Pol>(ky)] = in[(size_t)ky * nz + z];
    }
    __syncthreads();
    fft_lines<Pol, false, EMAX>(s, LS, sc, nl, tw, threadIdx.x, blockDim.x);
    for (int i = threadIdx.x; i < nl * ny; i += blockDim.x) {
        const int l = i / ny, y = i - l * ny;
        const int z = z0 + l;
        if (z < nz) W1[((size_t)z * hx + kx) * ny + y] = s[l * LS + pidx<Pol>(y)];
    }
}

// ------------------------------------------------------------------ pass xi
template <class Pol, int EMAX>
__global__ void __launch_bounds__(kMaxThreads) k_xi(const S_t<Pol> *__restrict__ W1, typename Pol::io_t *__restrict__ u,
                                             int nx, int ny, int hx, Sched sc, int nl,
                                             const typename Pol::tw_t *__restrict__ tw)
{
    using R = typename Pol::real;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    S_t<Pol> *s = reinterpret_cast<S_t<Pol> *>(smem_raw);
    const int M = sc.M, LS = line_stride<Pol>(M);
    const int z = blockIdx.y;
    const int y0 = blockIdx.x * 2 * nl;
    const S_t<Pol> *in = W1 + (size_t)z * hx * ny;
    // Z[k] = A[k] + i B[k] (k = 0..nx), Z[M-k] = conj A[k] + i conj B[k];
    // A, B real at k = 0 and k = nx (DC and Nyquist of real rows)
    for (int i = threadIdx.x; i < hx * nl; i += blockDim.x) {
        const int k = i / nl, l = i - k * nl;
        const int ya = y0 + 2 * l;
        cx<R> A = {Pol::zero(), Pol::zero()}, B = {Pol::zero(), Pol::zero()};
        if (ya < ny) A = Pol::ld(in[(size_t)k * ny + ya]);
        if (ya + 1 < ny) B = Pol::ld(in[(size_t)k * ny + ya + 1]);
        if (k == 0 || k == nx) {
            A.im = Pol::zero();
            B.im = Pol::zero();
        }
        s[l * LS + pidx<Pol>(k)] = Pol::st(cadd(A, cmul_posi(B)));
        if (k > 0 && k < nx) s[l * LS + pidx<Pol>(M - k)] = Pol::st(cadd(cconj(A), cmul_posi(cconj(B))));
    }
    __syncthreads();
    fft_lines<Pol, false, EMAX>(s, LS, sc, nl, tw, threadIdx.x, blockDim.x);
    typename Pol::io_t *slab = u + (size_t)z * ny * nx;
    for (int i = threadIdx.x; i < nl * nx; i += blockDim.x) {
        const int l = i / nx, x = i - l * nx;
        const int ya = y0 + 2 * l;
        const cx<R> c = Pol::ld(s[l * LS + pidx<Pol>(x)]);
        if (ya < ny) slab[(size_t)ya * nx + x] = Pol::to_io(c.re);
        if (ya + 1 < ny) slab[(size_t)(ya + 1) * nx + x] = Pol::to_io(c.im);
    }
}

// ------------------------------------------------------------------ FFT test hook
template <class Pol, bool FWD, int EMAX>
__global__ void __launch_bounds__(kMaxThreads) k_fft_hook(const double2 *__restrict__ in, double2 *__restrict__ out,
                                                   int nlines, Sched sc, int nl,
                                                   const typename Pol::tw_t *__restrict__ tw)
{
    using R = typename Pol::real;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    S_t<Pol> *s = reinterpret_cast<S_t<Pol> *>(smem_raw);
    const int M = sc.M, LS = line_stride<Pol>(M);
    const int line0 = blockIdx.x * nl;
    for (int i = threadIdx.x; i < nl * M; i += blockDim.x) {
        const int l = i / M, k = i - l * M;
        double2 v = make_double2(0.0, 0.0);
        if (line0 + l < nlines) v = in[(size_t)(line0 + l) * M + k];
        s[l * LS + pidx<Pol>(k)] =
            Pol::st(cx<R>{Pol::from_io((typename Pol::io_t)v.x), Pol::from_io((typename Pol::io_t)v.y)});
    }
    __syncthreads();
    fft_lines<Pol, FWD, EMAX>(s, LS, sc, nl, tw, threadIdx.x, blockDim.x);
    for (int i = threadIdx.x; i < nl * M; i += blockDim.x) {
        const int l = i / M, k = i - l * M;
        if (line0 + l < nlines) {
            const cx<R> c = Pol::ld(s[l * LS + pidx<Pol>(k)]);
            out[(size_t)(line0 + l) * M + k] = make_double2((double)Pol::to_io(c.re), (double)Pol::to_io(c.im));
        }
    }
}

// ------------------------------------------------------------------ tables
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

// nl lines of length M per CTA, nthr threads, emax = elements per thread
// (8 or 16); nthr * emax >= nl * M.
template <class Pol>
PassCfg choose_cfg(int M, int nl_want)
{
    PassCfg c;
    int nl = std::max(1, nl_want);
    const size_t smem_cap = 200 * 1024;
    while (nl > 1 && (pass_smem<Pol>(M, nl) > smem_cap || (long)nl * M / 16 > kMaxThreads)) nl /= 2;
    int emax = ((long)nl * M / 8 <= kMaxThreads) ? 8 : 16;
    int nthr = (nl * M + emax - 1) / emax;
    nthr = ((nthr + 31) / 32) * 32;
    nthr = std::max(32, std::min(kMaxThreads, nthr));
    c.nl = nl;
    c.nthr = nthr;
    c.emax = emax;
    c.smem = pass_smem<Pol>(M, nl);
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
        p->cfg_conv = choose_cfg<Pol>(p->M[2], std::max(1, 4096 / p->M[2]));
    } else {
        p->cfg_conv = choose_cfg<Pol>(p->M[1], std::max(1, 4096 / p->M[1]));
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
    GSM_CUDA_TRY(cudaMalloc(&p->d_work1, p->work1_bytes));
    if (p->work2_bytes) GSM_CUDA_TRY(cudaMalloc(&p->d_work2, p->work2_bytes));
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
    const int last = p->d == 3 ? 4 : 2;
    if (pass == 0) {
        const PassCfg &c = p->cfg_xf;
        dim3 g((ny + 2 * c.nl - 1) / (2 * c.nl), nz);
        with_emax(c, [&](auto E) {
            k_xf<Pol, E()><<<g, c.nthr, c.smem, st>>>(rho, W1, nx, ny, hx, p->sched[0], c.nl, twx);
        });
    } else if (pass == last) {
        const PassCfg &c = p->cfg_xi;
        dim3 g((ny + 2 * c.nl - 1) / (2 * c.nl), nz);
        with_emax(c, [&](auto E) {
            k_xi<Pol, E()><<<g, c.nthr, c.smem, st>>>(W1, u, nx, ny, hx, p->sched[0], c.nl, twx);
        });
    } else if (p->d == 2) {
        const PassCfg &c = p->cfg_conv;
        with_emax(c, [&](auto E) {
            k_conv<Pol, E()><<<(hx + c.nl - 1) / c.nl, c.nthr, c.smem, st>>>(W1, mult, hx, ny, 0, 1, ny + 1,
                                                                          p->sched[1], c.nl, twy);
        });
    } else {
        const tw *twz = static_cast<const tw *>(p->d_tw[2]);
        const int My = p->M[1];
        if (pass == 1) {
            const PassCfg &c = p->cfg_yf;
            dim3 g((nz + c.nl - 1) / c.nl, hx);
            with_emax(c, [&](auto E) {
                k_yf<Pol, E()><<<g, c.nthr, c.smem, st>>>(W1, W2, ny, nz, hx, p->sched[1], c.nl, twy);
            });
        } else if (pass == 2) {
            const PassCfg &c = p->cfg_conv;
            const int nlines = hx * My;
            with_emax(c, [&](auto E) {
                k_conv<Pol, E()><<<(nlines + c.nl - 1) / c.nl, c.nthr, c.smem, st>>>(
                    W2, mult, nlines, nz, 1, My, ny + 1, p->sched[2], c.nl, twz);
            });
        } else {
            const PassCfg &c = p->cfg_yi;
            dim3 g((nz + c.nl - 1) / c.nl, hx);
            with_emax(c, [&](auto E) {
                k_yi<Pol, E()><<<g, c.nthr, c.smem, st>>>(W2, W1, ny, nz, hx, p->sched[1], c.nl, twy);
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

template <class Pol>
gsm_status_t fft_hook_t(int M, int nlines, int sign, const double *in, double *out, cudaStream_t st)
{
    Sched sc;
    if (!make_sched(M, &sc)) {
        set_error("FFT length must be a product of 2, 3, 5 between 2 and 8192");
        return GSM_ERR_UNSUPPORTED_SIZE;
    }
    void *d_tw = nullptr;
    GSM_CUDA_TRY(cudaMallocAsync(&d_tw, sizeof(typename Pol::tw_t) * M, st));
    k_twiddles<<<(M + 255) / 256, 256, 0, st>>>(M, Pol::kId, d_tw);
    const PassCfg c = choose_cfg<Pol>(M, std::max(1, 2048 / M));
    const auto *tw = static_cast<const typename Pol::tw_t *>(d_tw);
    const int blocks = (nlines + c.nl - 1) / c.nl;
    cudaError_t e = cudaSuccess;
    with_emax(c, [&](auto E) {
        if (sign < 0) {
            e = raise_smem(k_fft_hook<Pol, true, E()>, c.smem);
            if (e == cudaSuccess)
                k_fft_hook<Pol, true, E()><<<blocks, c.nthr, c.smem, st>>>((const double2 *)in, (double2 *)out,
                                                                           nlines, sc, c.nl, tw);
        } else {
            e = raise_smem(k_fft_hook<Pol, false, E()>, c.smem);
            if (e == cudaSuccess)
                k_fft_hook<Pol, false, E()><<<blocks, c.nthr, c.smem, st>>>((const double2 *)in, (double2 *)out,
                                                                            nlines, sc, c.nl, tw);
        }
    });
    GSM_CUDA_TRY(e);
    GSM_CUDA_TRY(cudaGetLastError());
    GSM_CUDA_TRY(cudaFreeAsync(d_tw, st));
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

gsm_status_t make_twiddles(Plan *p, int axis, cudaStream_t st)
{
    for (int b = 0; b < axis; ++b)
        if (p->M[b] == p->M[axis]) {
            p->d_tw[axis] = p->d_tw[b];
            return GSM_OK;
        }
    const int M = p->M[axis];
    GSM_CUDA_TRY(cudaMalloc(&p->d_tw[axis], cplx_bytes(p->opt.precision) * M));
    k_twiddles<<<(M + 255) / 256, 256, 0, st>>>(M, p->opt.precision, p->d_tw[axis]);
    GSM_CUDA_TRY(cudaGetLastError());
    return GSM_OK;
}

gsm_status_t make_pass_multiplier(Plan *p, cudaStream_t st)
{
    if (p->opt.precision == GSM_FP64) {
        p->d_mult = p->d_mult64;
        return GSM_OK;
    }
    const size_t eb = p->opt.precision == GSM_FP32 ? sizeof(float) : sizeof(float2);
    GSM_CUDA_TRY(cudaMalloc(&p->d_mult, eb * p->mult_elems));
    k_mult_convert<<<(p->mult_elems + 255) / 256, 256, 0, st>>>(p->d_mult64, p->mult_elems, p->opt.precision,
                                                                  p->d_mult);
    GSM_CUDA_TRY(cudaGetLastError());
    return GSM_OK;
}

gsm_status_t configure_passes(Plan *p)
{
    for (int a = 0; a < p->d; ++a)
        if (!make_sched(p->M[a], &p->sched[a])) {
            set_error("padded length 2n must be a product of 2, 3 and 5");
            return GSM_ERR_UNSUPPORTED_SIZE;
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

gsm_status_t launch_pass(const Plan *p, int pass, const void *rho, void *u, cudaStream_t st)
{
    switch (p->opt.precision) {
    case GSM_FP64: return pass_t<F64>(p, pass, rho, u, st);
    case GSM_FP32: return pass_t<F32>(p, pass, rho, u, st);
    default: return pass_t<DF64>(p, pass, rho, u, st);
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
        cell *= 2.0 * p->L / p->n[a];
    }
    if (!p->d_scratch) {
        GSM_CUDA_TRY(cudaMalloc(&p->d_scratch, sizeof(double) * kEnergyBlocks));
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
// Scratch of gsm_fft_lines_noalloc: the twiddle table of one transform length,
// up to 8192 entries of 16 bytes (FP64 or double-float pairs).  A file-scope
// __device__ array, so every GPU that loads this library holds these 128 KiB
// until the process exits; every call shares it.
namespace {

constexpr size_t kStaticTwiddleBytes = 8192 * 16;
__device__ __align__(256) unsigned char g_static_twiddles[kStaticTwiddleBytes];

constexpr int kMaxDevices = 64;
std::mutex g_static_mutex;
void *g_static_addr[kMaxDevices] = {};

// The host-side name g_static_twiddles is not a device address; the device
// address is looked up once per device, with that device current.
cudaError_t static_twiddle_address(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_static_mutex);
    if (!g_static_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_twiddles);
        if (e != cudaSuccess) return e;
        g_static_addr[dev] = p;
    }
    *out = g_static_addr[dev];
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
    if (sizeof(typename Pol::tw_t) * (size_t)M > kStaticTwiddleBytes) {
        set_error("FFT length exceeds the 128 KiB static twiddle scratch (M <= 8192)");
        return GSM_ERR_UNSUPPORTED_SIZE;
    }
    void *d_tw = nullptr;
    GSM_CUDA_TRY(static_twiddle_address(&d_tw));
    // every entry the FFT reads is written here first: nothing needs clearing
    k_twiddles<<<(M + 255) / 256, 256, 0, st>>>(M, Pol::kId, d_tw);
    const PassCfg c = choose_cfg<Pol>(M, std::max(1, 2048 / M));
    const auto *tw = static_cast<const typename Pol::tw_t *>(d_tw);
    const int blocks = (nlines + c.nl - 1) / c.nl;
    cudaError_t e = cudaSuccess;
    with_emax(c, [&](auto E) {
        if (sign < 0) {
            e = raise_smem(k_fft_hook<Pol, true, E()>, c.smem);
            if (e == cudaSuccess)
                k_fft_hook<Pol, true, E()><<<blocks, c.nthr, c.smem, st>>>((const double2 *)in, (double2 *)out,
                                                                           nlines, sc, c.nl, tw);
        } else {
            e = raise_smem(k_fft_hook<Pol, false, E()>, c.smem);
            if (e == cudaSuccess)
                k_fft_hook<Pol, false, E()><<<blocks, c.nthr, c.smem, st>>>((const double2 *)in, (double2 *)out,
                                                                            nlines, sc, c.nl, tw);
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

}  // namespace gsm
