// gsm_tc.cu -- a 32-point DFT stage on the tensor cores (tcgen05) with
// FP64-class accuracy, built to measure whether tensor-core DFT stages can
// serve the FP64-class passes of the method (Eq. I1FFT) on GB300.
//
// A stage of an FFT is a batch of small DFTs, a dense product: for vectors x
// (32 complex values, 64 reals: the real parts, then the imaginary parts) the
// DFT is Y = F x with F the 64 x 64 real form of the DFT matrix.  The tensor
// cores multiply bf16 values (8 significant bits) exactly and accumulate in
// FP32, so each FP64 operand is split into digits first (the splitting scheme
// of K. Ozaki, T. Ogita, S. Oishi and S. M. Rump, "Error-free transformations
// of matrix multiplication by using fast routines of matrix multiplication",
// Numer. Algorithms 59 (2012)):
//   - every vector is scaled by a power of two 2^e >= its largest |x|, and the
//     scaled value rounded to a 48-bit integer T (integer arithmetic on the
//     FP64 bit pattern), written as six balanced base-256 digits
//     T = sum_j d_j 256^(5-j), |d_j| <= 128 (exact in bf16);
//   - F's entries (|f| <= 1) the same way with e = 0.
// The product of digit planes i (of F) and j (of x) has the scale
// 2^(e - 14 - 8 (i + j)); the planes with i + j = s (s = 0..5, 21 products)
// accumulate into one FP32 accumulator per s in tensor memory.  Every partial
// sum is an integer below 6 * 64 * 128 * 128 < 2^23: exact in FP32.  The
// dropped planes (i + j >= 6) and the rounding of x and F to 48 bits leave
// an error of about 2^-47 of the vector's largest value per input, FP64-class
// (the double-float passes carry 48 bits).  The six levels are summed as a
// 64-bit integer (|sum| < 2^61) and converted to FP64 once.
//
// One CTA of 4 warps takes 128 vectors: the tensor-core product has M = 128
// (vectors, one per TMEM lane), N = 64 (output reals), K = 16 per instruction,
// 4 instructions per digit-plane product, 84 in all, issued by one thread;
// tcgen05.commit signals an mbarrier when they are done, and every thread
// reads its vector's six accumulators back with tcgen05.ld.
//
// Operands in shared memory, K-major without swizzle: 8-row x 16-byte core
// matrices; for K-chunk kc (16 reals) and row group rg, the two core matrices
// (reals 0-7 and 8-15 of the chunk) lie at chunk base + rg * 256 + {0, 128}:
// leading-dimension offset (K direction) 128 bytes, stride-dimension offset
// (rows) 256 bytes.
#include <cuda_bf16.h>

#include "gsm_internal.h"

namespace gsm {

namespace {

constexpr int kTcVecs = 128;        // vectors per CTA (the MMA's M)
constexpr int kTcK = 64;            // reals per vector (K), outputs per vector (N)
constexpr int kTcDigits = 6;        // base-256 digits per value (48 bits)
constexpr int kTcLevels = 6;        // accumulated levels s = i + j <= 5
constexpr int kTcChunkA = kTcVecs / 8 * 256;          // bytes of one K-chunk of x's digit plane
constexpr int kTcPlaneA = 4 * kTcChunkA;              // bytes of one digit plane of x (16 KB)
constexpr int kTcChunkB = kTcK / 8 * 256;             // one K-chunk of F's digit plane
constexpr int kTcPlaneB = 4 * kTcChunkB;              // one digit plane of F (8 KB)
constexpr int kTcSmemB = kTcDigits * kTcPlaneB;       // 48 KB
constexpr int kTcSmemA = kTcDigits * kTcPlaneA;       // 96 KB
constexpr int kTcSmem = kTcSmemB + kTcSmemA + 1024;   // + alignment slack
constexpr unsigned long long kTcWaitNs = 1000000000ull;   // bound of the MMA wait (1 s)

// Byte offset of element (row r, K index k) in a digit plane of `rows` rows.
__host__ __device__ __forceinline__ int tc_offset(int rows, int r, int k)
{
    const int kc = k >> 4, kh = (k >> 3) & 1, e = k & 7;
    return kc * (rows / 8 * 256) + (r >> 3) * 256 + kh * 128 + (r & 7) * 16 + e * 2;
}

// T = round(x 2^(47 - e)) as a signed integer, |x| <= 2^e; integer operations
// on the bit pattern (no FP64 arithmetic).
__device__ __forceinline__ long long tc_fixed(double x, int e)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int E = (int)((b >> 52) & 0x7ff);
    if (E == 0) return 0;   // zero or subnormal: below 2^-47 of any normal block scale
    const unsigned long long M = (b & 0xfffffffffffffull) | (1ull << 52);
    // x = M 2^(E - 1075); T = M 2^(E - 1075 + 47 - e) = M >> s
    const int s = 1028 + e - E;
    unsigned long long T;
    if (s <= 0) T = M << (-s);                 // not reached for |x| <= 2^e (s >= 6)
    else if (s > 62) T = 0;
    else T = (M + (1ull << (s - 1))) >> s;     // round half up on the magnitude
    return (b >> 63) ? -(long long)T : (long long)T;
}

// Six balanced base-256 digits of T (|T| <= 2^47): T = sum_j d[j] 256^(5 - j).
__device__ __forceinline__ void tc_digits(long long T, int *d)
{
#pragma unroll
    for (int j = kTcDigits - 1; j > 0; --j) {
        int v = (int)(T & 255);
        if (v >= 128) v -= 256;
        d[j] = v;
        T = (T - v) >> 8;
    }
    d[0] = (int)T;
}

// Digit planes of F (the real 64 x 64 DFT matrix of length 32, sign -1
// forward, +1 inverse) in the shared-memory layout, one thread per entry.
// Row n: outputs Re Y[n] (n < 32), Im Y[n - 32]; column k: Re x[k] (k < 32),
// Im x[k - 32].
__global__ void k_tc_ftable(int sign, __nv_bfloat16 *out)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= kTcK * kTcK) return;
    const int n = idx / kTcK, k = idx % kTcK;
    const int kk = n & 31, p = k & 31;
    double sn, cs;
    sincospi(2.0 * (double)((kk * p) & 31) / 32.0, &sn, &cs);
    const double s = sign < 0 ? sn : -sn;   // x w^(p kk), w = exp(sign 2 pi i / 32): Re = xr cs + xi s
    double f;
    if (n < 32) f = (k < 32) ? cs : s;
    else f = (k < 32) ? -s : cs;
    int d[kTcDigits];
    tc_digits(tc_fixed(f, 0), d);
    unsigned char *base = reinterpret_cast<unsigned char *>(out);
    for (int i = 0; i < kTcDigits; ++i)
        *reinterpret_cast<__nv_bfloat16 *>(base + i * kTcPlaneB + tc_offset(kTcK, n, k)) =
            __float2bfloat16_rn((float)d[i]);
}

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long tc_desc(unsigned saddr)
{
    // start address >> 4 (bits 0-13), leading-dimension offset 128 B >> 4 (bits 16-29),
    // stride-dimension offset 256 B >> 4 (bits 32-45), descriptor version 1 (bits 46-47),
    // base offset 0, no swizzle (bits 61-63 = 0)
    return (unsigned long long)((saddr >> 4) & 0x3fff) | ((unsigned long long)(128 >> 4) << 16) |
           ((unsigned long long)(256 >> 4) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: D FP32 (bits 4-5 = 1), A and B bf16
// (bits 7-9, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 (bits 17-22),
// M >> 4 (bits 24-28).
constexpr unsigned kTcIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(kTcK >> 3) << 17) |
                              ((unsigned)(kTcVecs >> 4) << 24);

__device__ __forceinline__ unsigned long long tc_global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for phase `parity` of the mbarrier, at most kTcWaitNs; false if the wait ran out.
__device__ __forceinline__ bool tc_wait(unsigned mbar, unsigned parity)
{
    const unsigned long long t0 = tc_global_ns();
    for (;;) {
        unsigned done;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done)
                     : "r"(mbar), "r"(parity)
                     : "memory");
        if (done) return true;
        if (tc_global_ns() - t0 > kTcWaitNs) return false;
        __nanosleep(64);
    }
}

__global__ void __launch_bounds__(kTcVecs, 1)
    k_dft32_tc(const double2 *__restrict__ in, double2 *__restrict__ out, int nvec,
               const __nv_bfloat16 *__restrict__ ftab, unsigned *status)
{
    extern __shared__ unsigned char tc_raw[];
    __shared__ __align__(8) unsigned long long mbar;
    __shared__ unsigned tmem_base;
    unsigned char *smem = reinterpret_cast<unsigned char *>(((size_t)tc_raw + 1023) & ~(size_t)1023);
    unsigned char *sB = smem;
    unsigned char *sA = smem + kTcSmemB;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int v = blockIdx.x * kTcVecs + tid;   // this thread's vector (= its row, = its TMEM lane)

    // tensor memory: 512 columns (6 accumulators of 64 columns), one warp allocates
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(&tmem_base))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // F's digit planes (48 KB, already in the shared layout)
    {
        const int4 *src = reinterpret_cast<const int4 *>(ftab);
        int4 *dst = reinterpret_cast<int4 *>(sB);
        for (int i = tid; i < kTcSmemB / 16; i += kTcVecs) dst[i] = src[i];
    }
    // this vector: scale 2^e > max|x|, digits of every real into the six planes
    // of x, eight reals (one 16-byte core-matrix row) per store
    int e_out = 0;
    {
        double2 x[32];
        double mx = 0.0;
#pragma unroll
        for (int p = 0; p < 32; ++p) {
            x[p] = v < nvec ? in[(size_t)v * 32 + p] : make_double2(0.0, 0.0);
            mx = fmax(mx, fmax(fabs(x[p].x), fabs(x[p].y)));
        }
        if (mx > 0.0) frexp(mx, &e_out);
#pragma unroll
        for (int g = 0; g < kTcK / 8; ++g) {
            unsigned w[kTcDigits][4];
#pragma unroll
            for (int q = 0; q < 8; q += 2) {
                const int k0 = 8 * g + q, k1 = k0 + 1;
                const double a0 = k0 < 32 ? x[k0].x : x[k0 - 32].y;
                const double a1 = k1 < 32 ? x[k1].x : x[k1 - 32].y;
                int d0[kTcDigits], d1[kTcDigits];
                tc_digits(tc_fixed(a0, e_out), d0);
                tc_digits(tc_fixed(a1, e_out), d1);
#pragma unroll
                for (int j = 0; j < kTcDigits; ++j) {
                    const __nv_bfloat162 h = __floats2bfloat162_rn((float)d0[j], (float)d1[j]);
                    w[j][q / 2] = *reinterpret_cast<const unsigned *>(&h);
                }
            }
            const int off = tc_offset(kTcVecs, tid, 8 * g);
#pragma unroll
            for (int j = 0; j < kTcDigits; ++j)
                *reinterpret_cast<uint4 *>(sA + j * kTcPlaneA + off) = make_uint4(w[j][0], w[j][1], w[j][2], w[j][3]);
        }
    }
    // generic-proxy writes of the operands, then visible to the tensor cores
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tmem = tmem_base;
    if (tid == 0) {
        const unsigned aBase = smem_u32(sA), bBase = smem_u32(sB);
        for (int s = 0; s < kTcLevels; ++s) {
            bool first = true;
            for (int i = 0; i <= s; ++i) {
                const int j = s - i;   // F plane i, x plane j
                for (int kc = 0; kc < 4; ++kc) {
                    const unsigned long long da = tc_desc(aBase + j * kTcPlaneA + kc * kTcChunkA);
                    const unsigned long long db = tc_desc(bBase + i * kTcPlaneB + kc * kTcChunkB);
                    const unsigned acc = first ? 0u : 1u;
                    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(
                                     tmem + (unsigned)(s * kTcK)),
                                 "l"(da), "l"(db), "r"(kTcIdesc), "r"(acc)
                                 : "memory");
                    first = false;
                }
            }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(&mbar))
                     : "memory");
    }
    bool ok = tc_wait(smem_u32(&mbar), 0);
    if (!ok) {
        if (tid == 0) atomicExch(status, (unsigned)GSM_ERR_TIMEOUT);
        ok = tc_wait(smem_u32(&mbar), 0);   // the products may still be running: wait once more
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) {
        // each warp reads its 32 lanes; per 16 output columns, the six levels
        const unsigned lane_base = tmem + ((unsigned)(warp * 32) << 16);
        double2 *o = out + (size_t)v * 32;
#pragma unroll 1
        for (int c = 0; c < kTcK / 16; ++c) {
            unsigned L[kTcLevels][16];
#pragma unroll
            for (int s = 0; s < kTcLevels; ++s) {
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
                    "%12, %13, %14, %15}, [%16];"
                    : "=r"(L[s][0]), "=r"(L[s][1]), "=r"(L[s][2]), "=r"(L[s][3]), "=r"(L[s][4]), "=r"(L[s][5]),
                      "=r"(L[s][6]), "=r"(L[s][7]), "=r"(L[s][8]), "=r"(L[s][9]), "=r"(L[s][10]), "=r"(L[s][11]),
                      "=r"(L[s][12]), "=r"(L[s][13]), "=r"(L[s][14]), "=r"(L[s][15])
                    : "r"(lane_base + (unsigned)(s * kTcK + c * 16)));
            }
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                // sum_s L_s 2^(8 (5 - s)), each L_s an integer held exactly in FP32
                long long acc = 0;
#pragma unroll
                for (int s = 0; s < kTcLevels; ++s)
                    acc += (long long)__float2ll_rn(__uint_as_float(L[s][q])) << (8 * (kTcLevels - 1 - s));
                // Y = acc 2^(e - 14 - 40): convert once, then set the exponent by integer
                // addition (y >= 1, so the sum is normal unless e is far below 0)
                double y = __ll2double_rn(acc);
                if (y != 0.0) {
                    const long long yb = __double_as_longlong(y);
                    const int biased = (int)((yb >> 52) & 0x7ff) + e_out - 54;
                    y = biased > 0 ? __longlong_as_double(yb + ((long long)(e_out - 54) << 52))
                                   : ldexp(y, e_out - 54);
                }
                const int n = c * 16 + q;
                if (v < nvec) {
                    if (n < 32) reinterpret_cast<double *>(o + n)[0] = y;
                    else reinterpret_cast<double *>(o + (n - 32))[1] = y;
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
}

}  // namespace

gsm_status_t launch_dft32_tc(int nvec, int sign, const double *in, double *out, cudaStream_t st)
{
    void *tab = nullptr, *stat = nullptr;
    GSM_CUDA_TRY(dev_alloc_async_bytes(&tab, kTcSmemB, st));
    cudaError_t e = dev_alloc_async_bytes(&stat, sizeof(unsigned), st);
    if (e != cudaSuccess) {
        dev_free_async(tab, st);
        GSM_CUDA_TRY(e);
    }
    e = cudaMemsetAsync(stat, 0, sizeof(unsigned), st);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_dft32_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem);
    if (e == cudaSuccess) {
        k_tc_ftable<<<(kTcK * kTcK + 255) / 256, 256, 0, st>>>(sign, static_cast<__nv_bfloat16 *>(tab));
        k_dft32_tc<<<(nvec + kTcVecs - 1) / kTcVecs, kTcVecs, kTcSmem, st>>>(
            reinterpret_cast<const double2 *>(in), reinterpret_cast<double2 *>(out), nvec,
            static_cast<const __nv_bfloat16 *>(tab), static_cast<unsigned *>(stat));
        e = cudaGetLastError();
    }
    unsigned h = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, stat, sizeof(h), cudaMemcpyDeviceToHost, st);
    dev_free_async(tab, st);
    dev_free_async(stat, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    GSM_CUDA_TRY(e);
    if (h != 0) {
        set_error("the tensor-core product's completion wait ran out");
        return GSM_ERR_TIMEOUT;
    }
    return GSM_OK;
}

}  // namespace gsm
