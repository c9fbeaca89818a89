// gsm_internal.h -- plan structure and internal entry points of the library.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <string>

#include "../../include/gsm.h"
#include "gsm_fft.cuh"

namespace gsm {

constexpr uint64_t kPlanMagic = 0x47534d504c414e31ull;   // "GSMPLAN1"
constexpr int kMaxM = 8192;
constexpr int kMinN = 8;
constexpr int kSmax = 500;          // largest sinc parameter S scanned by the plan
constexpr int kGsCap = 2 * kSmax + 2;

// Launch shape of one pass: nl lines of length M per CTA, each transformed
// by a group of gthr threads holding up to emax elements each; nthr = nl * gthr.
struct PassCfg {
    int nl = 1;
    int gthr = 256;
    int nthr = 256;
    int emax = 8;      // complex elements per thread (template instance)
    size_t smem = 0;
};

struct Plan {
    uint64_t magic = 0;
    gsm_kernel_t kind;
    int d = 3;
    int n[3] = {1, 1, 1};
    int M[3] = {1, 1, 1};
    double L = 1.0;                 // reference half-width (largest of the box)
    double eta[3] = {1.0, 1.0, 1.0};   // half-width of each axis in units of L (Sec. 2.5)
    double eps = 0.0;
    gsm_options_t opt;
    int device = 0;
    int dip_axis = -1;             // n and m both along this axis (octant multiplier)

    // plan results (Sec. 3, Sec. 2.3)
    int S = 0, nterms = 0;
    double gs_err = 0.0, c0 = 0.0, c2 = 0.0;

    // device data
    double *d_w = nullptr, *d_tau = nullptr;      // Gaussian sum
    double *d_g[3] = {nullptr, nullptr, nullptr}; // 1-D factors [q][k] per axis
    double *d_khat = nullptr;                     // sum_q w_q G_k^q, octant, FP64
    double *d_mult64 = nullptr;                   // full multiplier, FP64, octant
    void *d_mult = nullptr;                       // multiplier in the pass precision
    void *d_tw[3] = {nullptr, nullptr, nullptr};  // per axis: twiddles, then (FP64) the FMA-form
                                                  // constants of the forward schedule
    void *d_twi[3] = {nullptr, nullptr, nullptr}; // the same for the inverse schedule (may alias d_tw)
    void *d_work1 = nullptr, *d_work2 = nullptr;  // FFT workspace
    size_t work1_bytes = 0, work2_bytes = 0;
    size_t mult_elems = 0;         // octant entries (FP64 tables)
    size_t mult_elems_pass = 0;    // entries of the pass-precision table
    bool mult_full = false;        // pass table covers the half spectrum (general dipolar)
    bool rr_conv = true;           // FP32, padded length 512: the register-resident x, y, conv kernels
    void *d_stage_in = nullptr, *d_stage_out = nullptr;   // gsm_apply_host staging
    cudaStream_t copy_stream = nullptr;                    // gsm_apply_host copies (3D)
    cudaEvent_t copy_ev[2 * 8 + 2] = {};                   // chunk events of that pipeline
    double *d_scratch = nullptr;                           // energy partial sums
    size_t scratch_elems = 0;

    Sched sched_f[3], sched_i[3];   // radix schedules of the forward and inverse transforms per axis
    PassCfg cfg_xf, cfg_yf, cfg_conv, cfg_yi, cfg_xi;
    // 2D conv of padded length >= kSplitMinM: each line as two transforms of
    // half the length on a cluster of two CTAs (k_conv_split)
    bool split_conv = false;
    Sched sched_hf, sched_hi;
    void *d_twh = nullptr, *d_twhi = nullptr;   // tables of the half length
    PassCfg cfg_split;
    // 2D x forward pass of padded length >= kSplitMinM: each line as two
    // half-length transforms on two CTAs (k_xf_split)
    bool split_x = false;
    Sched sched_xh;                 // length M[0] / 2
    void *d_twxh = nullptr;         // its tables
    PassCfg cfg_xsplit;
};

// thread-local last error
void set_error(const std::string &msg);

// Every device allocation of the library goes through these functions (gsm_api.cu).
// They keep a count of what is live and can be told to fail (gsm_debug_fail_alloc),
// so that the clean-up on every out-of-memory path can be tested without
// exhausting a GPU.
cudaError_t dev_alloc_bytes(void **ptr, size_t bytes);
cudaError_t dev_alloc_async_bytes(void **ptr, size_t bytes, cudaStream_t st);
void dev_free(void *ptr);
void dev_free_async(void *ptr, cudaStream_t st);
template <class T>
inline cudaError_t dev_alloc(T **ptr, size_t bytes)
{
    return dev_alloc_bytes(reinterpret_cast<void **>(ptr), bytes);
}
// A temporary device buffer freed when it goes out of scope (dev_free waits
// for the device, as cudaFree does, so kernels still using it finish first).
struct DevTemp {
    void *p = nullptr;
    DevTemp() = default;
    DevTemp(const DevTemp &) = delete;
    DevTemp &operator=(const DevTemp &) = delete;
    ~DevTemp() { dev_free(p); }
    template <class T>
    T *as() const { return static_cast<T *>(p); }
};

// Precomputed results a saved plan carries (Sec. 2.2: the sum over q of
// w_q G_k^q is stored once per discretisation and reused).  Host arrays.
struct StoredPlanData {
    double L = 0.0, eta[3] = {1.0, 1.0, 1.0};    // box, exactly as saved
    int S = 0, nterms = 0;
    double gs_err = 0.0, c0 = 0.0, c2 = 0.0;
    const double *w = nullptr, *tau = nullptr;   // nterms each
    const double *khat = nullptr;                // octant tensor, mult_elems entries
};

// plan construction on the GPU (gsm_plan.cu); with stored != NULL the
// Gaussian sum, the Taylor coefficients and the kernel tensor are taken from
// it instead of being computed
gsm_status_t build_plan_data(Plan *p, cudaStream_t st, const StoredPlanData *stored = nullptr);

// passes (gsm_passes.cu)
gsm_status_t configure_passes(Plan *p);
gsm_status_t launch_apply(const Plan *p, const void *rho, void *u, cudaStream_t st);
gsm_status_t launch_pass(const Plan *p, int pass, const void *rho, void *u, cudaStream_t st);
// 3D only: the x forward pass (inverse = false, reads rho) or the x inverse
// pass (inverse = true, writes u) on the z-slabs [z0, z1); rho and u point
// at the whole arrays
gsm_status_t launch_x_slabs(const Plan *p, bool inverse, int z0, int z1, const void *rho, void *u,
                            cudaStream_t st);
constexpr int kHostChunks = 8;       // z-chunks of the pipelined host apply
// conv pass of FP32 plans with padded conv length 512, register-resident (gsm_conv_rr.cu)
gsm_status_t launch_conv_rr512_f32(void *W, const void *mult, int nlines, int is3d, int My, int ny1, bool full,
                                   const void *tw, cudaStream_t st);
// y passes of 3D FP32 plans with ny = 256 (forward W1 -> W2, inverse W2 -> W1), register-resident
gsm_status_t launch_y_rr512_f32(bool inverse, const void *in, void *out, int nz, int hx, const void *tw,
                                cudaStream_t st);
// x passes of FP32 plans with nx = 256 on nz slabs (forward rho -> W1, inverse W1 -> u)
gsm_status_t launch_x_rr512_f32(bool inverse, const void *in, void *out, int ny, int nz, const void *tw,
                                cudaStream_t st);
gsm_status_t autotune_plan(Plan *p, cudaStream_t st, std::string *report);
// set the launch shape of one pass (nl lines per CTA, emax elements per thread)
gsm_status_t set_pass_shape(Plan *p, int pass, int nl, int emax);
// The batched apply (gsm_passes.cu): plans with all padded lengths <= 512 go
// through one queue launch per (precision, dimension) group, whose
// work-queue state lives at `state` (batch_state_bytes(count) bytes of device
// memory, zeroed by the call); the others are applied one by one.  dry: only
// prepare the kernels.  batch_status reads the state after the stream's work:
// GSM_ERR_TIMEOUT if a bounded wait ran out.
gsm_status_t launch_batched(int count, const Plan *const *plans, const void *const *rho, void *const *u,
                            int nl, cudaStream_t st, bool dry, unsigned *state);
size_t batch_state_bytes(int count);
gsm_status_t batch_status(const unsigned *state, int count, cudaStream_t st);
// Bound of every wait of the batch queue kernel (0: the default) and the
// test hook that keeps one instance's first pass from ever counting as
// complete (-1: off); read when a batch is launched or recorded.
void set_batch_wait(unsigned long long wait_ns, int hold);
constexpr unsigned long long kBatchWaitDefaultNs = 10000000000ull;   // 10 s
constexpr int kBatchLines = 4;      // default lines (warps) per CTA of the batch queue kernel
constexpr int kBatchMaxLines = 8;   // largest shape tried (bounds the CTA size)
gsm_status_t launch_hartree(Plan *p, const void *psi, void *u, void *energy, void *grad,
                            cudaStream_t st);
gsm_status_t launch_fft_lines(int M, int nlines, int sign, gsm_precision_t prec,
                              const double *in, double *out, cudaStream_t st);
gsm_status_t launch_fft_lines_noalloc(int M, int nlines, int sign, gsm_precision_t prec,
                                      const double *in, double *out, cudaStream_t st);
// length-32 DFTs on the tensor cores (gsm_tc.cu); synchronises the stream
gsm_status_t launch_dft32_tc(int nvec, int sign, const double *in, double *out, cudaStream_t st);
// the twiddle tables of one axis for its current forward and inverse schedules
// (frees the axis's previous tables unless another axis shares them)
gsm_status_t make_twiddles(Plan *p, int axis, cudaStream_t st);
gsm_status_t make_pass_multiplier(Plan *p, cudaStream_t st);
// default radix schedule of length M: radices 8, 4, 2, 5, 3 in that order
bool make_sched(int M, Sched *s);
constexpr int kSplitMinM = 4096;
// the half-length schedules and tables of a split 2D conv (gsm_passes.cu)
gsm_status_t make_split_tables(Plan *p, cudaStream_t st);
gsm_status_t make_xsplit_tables(Plan *p, cudaStream_t st);
// schedule with the given radices in the given order (each 8, 4, 2, 5 or 3,
// product M); forward: the first radix must be even (the pruned first stage
// of a zero-padded transform)
bool make_sched_order(int M, const int *radices, int count, bool forward, Sched *s);
// set the schedule of one axis and direction, or both, and rebuild that axis's tables
gsm_status_t set_axis_schedule(Plan *p, int axis, bool inverse, const Sched &sc, cudaStream_t st);
gsm_status_t set_axis_pair(Plan *p, int axis, const Sched &f, const Sched &i, cudaStream_t st);
// whether a (forward, inverse) pair of schedules can run on the axis
bool axis_pair_ok(const Plan *p, int axis, const Sched &f, const Sched &i);
size_t cplx_bytes(gsm_precision_t prec);

}  // namespace gsm

#define GSM_CUDA_TRY(call)                                                                  \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess) {                                                            \
            gsm::set_error(std::string(#call) + ": " + cudaGetErrorString(e_));             \
            return e_ == cudaErrorMemoryAllocation ? GSM_ERR_OOM : GSM_ERR_CUDA;            \
        }                                                                                   \
    } while (0)
