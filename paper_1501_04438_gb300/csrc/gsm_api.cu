// gsm_api.cu -- the C interface declared in include/gsm.h.
#include <math.h>
#include <string.h>

#include <atomic>
#include <mutex>
#include <new>
#include <string>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "gsm_internal.h"

namespace gsm {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

// ---------------------------------------------------------------- device allocations
// Live allocations (address -> bytes) and the injected failure: g_fail_in > 0
// counts allocations down to the one that fails; 0 fails the next; < 0 is off.
static std::mutex g_alloc_mutex;
static std::unordered_map<void *, size_t> g_alloc_live;
static size_t g_alloc_bytes = 0;
static std::atomic<long> g_fail_in{-1};

static bool injected_failure()
{
    long k = g_fail_in.load();
    while (k >= 0) {
        if (g_fail_in.compare_exchange_weak(k, k - 1)) return k == 0;
    }
    return false;
}

static void track(void *ptr, size_t bytes)
{
    std::lock_guard<std::mutex> lock(g_alloc_mutex);
    g_alloc_live[ptr] = bytes;
    g_alloc_bytes += bytes;
}

static bool untrack(void *ptr)
{
    std::lock_guard<std::mutex> lock(g_alloc_mutex);
    auto it = g_alloc_live.find(ptr);
    if (it == g_alloc_live.end()) return false;
    g_alloc_bytes -= it->second;
    g_alloc_live.erase(it);
    return true;
}

cudaError_t dev_alloc_bytes(void **ptr, size_t bytes)
{
    *ptr = nullptr;
    if (injected_failure()) return cudaErrorMemoryAllocation;
    cudaError_t e = cudaMalloc(ptr, bytes);
    if (e != cudaSuccess) {
        *ptr = nullptr;
        return e;
    }
    track(*ptr, bytes);
    return cudaSuccess;
}

cudaError_t dev_alloc_async_bytes(void **ptr, size_t bytes, cudaStream_t st)
{
    *ptr = nullptr;
    if (injected_failure()) return cudaErrorMemoryAllocation;
    cudaError_t e = cudaMallocAsync(ptr, bytes, st);
    if (e != cudaSuccess) {
        *ptr = nullptr;
        return e;
    }
    track(*ptr, bytes);
    return cudaSuccess;
}

void dev_free(void *ptr)
{
    if (ptr && untrack(ptr)) cudaFree(ptr);
}

void dev_free_async(void *ptr, cudaStream_t st)
{
    if (ptr && untrack(ptr)) cudaFreeAsync(ptr, st);
}

// ---------------------------------------------------------------- live handles
// A handle is valid while it is in this registry: gsm_plan / gsm_plan_load and
// gsm_batch_create add it, the destroy calls remove it before freeing, so a
// destroyed handle is rejected without its memory being read.
static std::mutex g_handle_mutex;
static std::unordered_set<const void *> g_live_plans, g_live_batches;

static void register_handle(std::unordered_set<const void *> &set, const void *h)
{
    std::lock_guard<std::mutex> lock(g_handle_mutex);
    set.insert(h);
}

static bool release_handle(std::unordered_set<const void *> &set, const void *h)
{
    std::lock_guard<std::mutex> lock(g_handle_mutex);
    return set.erase(h) != 0;
}

static bool is_live(const std::unordered_set<const void *> &set, const void *h)
{
    std::lock_guard<std::mutex> lock(g_handle_mutex);
    return h != nullptr && set.count(h) != 0;
}

static Plan *checked(gsm_plan_t h)
{
    if (!is_live(g_live_plans, h)) return nullptr;
    Plan *p = reinterpret_cast<Plan *>(h);
    return p->magic == kPlanMagic ? p : nullptr;
}

static void free_plan(Plan *p)
{
    if (!p) return;
    dev_free(p->d_w);
    dev_free(p->d_tau);
    for (int a = 0; a < 3; ++a) {
        bool dup = false;
        for (int b = 0; b < a; ++b) dup |= (p->d_g[b] == p->d_g[a]);
        if (!dup) dev_free(p->d_g[a]);
    }
    {
        void *tabs[6] = {p->d_tw[0], p->d_tw[1], p->d_tw[2], p->d_twi[0], p->d_twi[1], p->d_twi[2]};
        for (int a = 0; a < 6; ++a) {
            bool dup = false;
            for (int b = 0; b < a; ++b) dup |= (tabs[b] == tabs[a]);
            if (!dup) dev_free(tabs[a]);
        }
    }
    if (p->d_twhi != p->d_twh) dev_free(p->d_twhi);
    dev_free(p->d_twh);
    dev_free(p->d_twxh);
    dev_free(p->d_khat);
    if (p->d_mult != p->d_mult64) dev_free(p->d_mult);
    dev_free(p->d_mult64);
    dev_free(p->d_work1);
    dev_free(p->d_work2);
    dev_free(p->d_stage_in);
    dev_free(p->d_stage_out);
    for (cudaEvent_t e : p->copy_ev)
        if (e) cudaEventDestroy(e);
    if (p->copy_stream) cudaStreamDestroy(p->copy_stream);
    dev_free(p->d_scratch);
    p->magic = 0;
    delete p;
}

static size_t io_bytes(const Plan *p) { return p->opt.precision == GSM_FP32 ? sizeof(float) : sizeof(double); }

static size_t grid_points(const Plan *p)
{
    size_t N = 1;
    for (int a = 0; a < p->d; ++a) N *= (size_t)p->n[a];
    return N;
}

}  // namespace gsm

using namespace gsm;

extern "C" {

void gsm_default_options(gsm_options_t *opt)
{
    if (!opt) return;
    memset(opt, 0, sizeof(*opt));
    opt->delta = 1e-3;
    opt->S = 0;
    opt->precision = GSM_FP64;
    opt->dip_n[2] = 1.0;
    opt->dip_m[2] = 1.0;
    opt->debug = 0;
    opt->beta = 1.0;
    opt->host_zero_copy = 1;
}

const char *gsm_status_string(gsm_status_t s)
{
    switch (s) {
    case GSM_OK: return "ok";
    case GSM_ERR_INVALID_ARG: return "invalid argument";
    case GSM_ERR_UNSUPPORTED_SIZE: return "unsupported size";
    case GSM_ERR_OOM: return "out of device memory";
    case GSM_ERR_CUDA: return "CUDA error";
    case GSM_ERR_ACCURACY: return "Gaussian-sum accuracy not reachable";
    case GSM_ERR_TIMEOUT: return "device wait timed out";
    case GSM_ERR_BAD_PLAN: return "bad plan handle";
    }
    return "unknown status";
}

const char *gsm_last_error(void) { return g_last_error.c_str(); }

static gsm_status_t create_plan(gsm_plan_t *out, gsm_kernel_t kind, int d, double L, const int *n, double gs_eps,
                                const gsm_options_t *opt, void *cuda_stream, const StoredPlanData *stored)
{
    if (!out) {
        set_error("out is NULL");
        return GSM_ERR_INVALID_ARG;
    }
    *out = nullptr;
    if (kind < GSM_COULOMB_3D || kind > GSM_POWER_2D) {
        set_error("unknown kernel");
        return GSM_ERR_INVALID_ARG;
    }
    const int want_d = (kind == GSM_COULOMB_3D || kind == GSM_DIPOLAR_3D || kind == GSM_POWER_3D) ? 3 : 2;
    if (d != want_d) {
        set_error("dimension does not match the kernel");
        return GSM_ERR_INVALID_ARG;
    }
    gsm_options_t o;
    if (opt) o = *opt;
    else gsm_default_options(&o);
    // rectangular box (Sec. 2.5): rescale by the largest half-width
    double eta[3] = {1.0, 1.0, 1.0};
    int nbox = 0;
    for (int a = 0; a < d; ++a) nbox += o.box[a] != 0.0;
    if (nbox != 0) {
        double Lr = 0.0;
        for (int a = 0; a < d; ++a) {
            if (!(o.box[a] > 0.0) || !isfinite(o.box[a])) {
                set_error("options.box must give d positive finite half-widths (or all 0)");
                return GSM_ERR_INVALID_ARG;
            }
            Lr = fmax(Lr, o.box[a]);
        }
        for (int a = 0; a < d; ++a) eta[a] = o.box[a] / Lr;
        L = Lr;
    }
    if (!n || !(L > 0.0) || !isfinite(L)) {
        set_error("n is NULL or L is not a positive finite number");
        return GSM_ERR_INVALID_ARG;
    }
    if (!(o.delta > 0.0) || o.delta >= 0.5) {
        set_error("options.delta must be in (0, 0.5)");
        return GSM_ERR_INVALID_ARG;
    }
    if (stored) {
        // the box exactly as saved (L eta_a / L need not round back to eta_a)
        L = stored->L;
        for (int a = 0; a < d; ++a) eta[a] = stored->eta[a];
    }
    for (int a = 0; a < d; ++a)
        if (!(o.delta < eta[a])) {
            set_error("options.delta must be smaller than every box half-width / the largest (Sec. 2.5)");
            return GSM_ERR_INVALID_ARG;
        }
    if ((kind == GSM_POWER_3D || kind == GSM_POWER_2D) && !(o.beta > 0.0 && o.beta < d)) {
        set_error("options.beta must lie in (0, d) for the power kernels");
        return GSM_ERR_INVALID_ARG;
    }
    if (o.precision < GSM_FP64 || o.precision > GSM_FP32X2) {
        set_error("unknown precision");
        return GSM_ERR_INVALID_ARG;
    }
    for (int a = 0; a < d; ++a) {
        Sched sc;
        if (n[a] < kMinN || (n[a] & 1) || 2 * n[a] > kMaxM || !make_sched(2 * n[a], &sc)) {
            set_error("each n must be even, >= 8, with 2n <= 8192 a product of 2, 3 and 5");
            return GSM_ERR_UNSUPPORTED_SIZE;
        }
    }
    int dip_axis = -1;
    if (kind == GSM_DIPOLAR_3D) {
        double nn = 0, mm = 0;
        for (int a = 0; a < 3; ++a) {
            nn += o.dip_n[a] * o.dip_n[a];
            mm += o.dip_m[a] * o.dip_m[a];
        }
        if (!(fabs(nn - 1.0) < 1e-12) || !(fabs(mm - 1.0) < 1e-12)) {
            set_error("dipolar n and m must be unit vectors");
            return GSM_ERR_INVALID_ARG;
        }
        // n and m along one axis: the multiplier folds onto the octant;
        // otherwise a half-spectrum table is built (dip_axis = -1)
        for (int a = 0; a < 3; ++a)
            if (fabs(fabs(o.dip_n[a]) - 1.0) == 0.0 && fabs(fabs(o.dip_m[a]) - 1.0) == 0.0) dip_axis = a;
    }
    Plan *p = new (std::nothrow) Plan();
    if (!p) {
        set_error("host allocation failed");
        return GSM_ERR_OOM;
    }
    p->kind = kind;
    p->d = d;
    for (int a = 0; a < d; ++a) {
        p->n[a] = n[a];
        p->M[a] = 2 * n[a];
    }
    p->L = L;
    for (int a = 0; a < 3; ++a) p->eta[a] = eta[a];
    p->opt = o;
    p->rr_conv = (o.debug & 1) == 0;
    p->dip_axis = dip_axis;
    const bool log_kernel = kind == GSM_POISSON_2D || kind == GSM_DAVEY_STEWARTSON_2D;
    p->eps = gs_eps > 0.0 ? gs_eps : (log_kernel ? 1e-13 : 2e-15);
    cudaGetDevice(&p->device);
    p->magic = kPlanMagic;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    gsm_status_t s = configure_passes(p);
    if (s == GSM_OK) s = build_plan_data(p, st, stored);
    if (s != GSM_OK) {
        free_plan(p);
        return s;
    }
    register_handle(g_live_plans, p);
    *out = reinterpret_cast<gsm_plan_t>(p);
    return GSM_OK;
}

gsm_status_t gsm_plan(gsm_plan_t *out, gsm_kernel_t kind, int d, double L, const int *n, double gs_eps,
                      const gsm_options_t *opt, void *cuda_stream)
{
    return create_plan(out, kind, d, L, n, gs_eps, opt, cuda_stream, nullptr);
}

// ---------------------------------------------------------------- save / load
// Layout (native little-endian, both supported hosts): a fixed header, the
// Gaussian sum (w, tau), the FP64 octant kernel tensor, then a 64-bit FNV-1a
// checksum of everything before it.
static const uint64_t kSaveMagic = 0x47534d5341564531ull;   // "GSMSAVE1"
static const uint32_t kSaveVersion = 3;

struct SaveHeader {
    uint64_t magic;
    uint32_t version, header_bytes;
    int32_t kind, d, n[3], precision, S, nterms, npasses, nl[5], emax[5], pad_;
    double L, eta[3], eps, delta, dip_n[3], dip_m[3], gs_err, c0, c2, beta;
    uint64_t mult_elems;
    uint8_t radix[2][3][kMaxStages];   // forward, inverse radices per axis (0 after the last)
};
static_assert(sizeof(SaveHeader) % 8 == 0, "the arrays after the header stay 8-byte aligned");

static uint64_t fnv1a(const unsigned char *b, size_t len)
{
    uint64_t h = 14695981039346656037ull;
    for (size_t i = 0; i < len; ++i) {
        h ^= b[i];
        h *= 1099511628211ull;
    }
    return h;
}

gsm_status_t gsm_plan_save(gsm_plan_t h, void *buf, size_t capacity, size_t *bytes)
{
    Plan *p = checked(h);
    if (!p) {
        set_error("bad plan handle");
        return GSM_ERR_BAD_PLAN;
    }
    if (!bytes) {
        set_error("bytes is NULL");
        return GSM_ERR_INVALID_ARG;
    }
    const size_t need = sizeof(SaveHeader) + sizeof(double) * (2 * (size_t)p->nterms + p->mult_elems) +
                        sizeof(uint64_t);
    *bytes = need;
    if (!buf) return GSM_OK;
    if (capacity < need) {
        set_error("buffer smaller than the saved plan (query the size with buf = NULL)");
        return GSM_ERR_INVALID_ARG;
    }
    SaveHeader hd;
    memset(&hd, 0, sizeof(hd));
    hd.magic = kSaveMagic;
    hd.version = kSaveVersion;
    hd.header_bytes = sizeof(SaveHeader);
    hd.kind = p->kind;
    hd.d = p->d;
    for (int a = 0; a < 3; ++a) {
        hd.n[a] = a < p->d ? p->n[a] : 1;
        hd.eta[a] = p->eta[a];
        hd.dip_n[a] = p->opt.dip_n[a];
        hd.dip_m[a] = p->opt.dip_m[a];
    }
    hd.precision = p->opt.precision;
    hd.S = p->S;
    hd.nterms = p->nterms;
    hd.npasses = p->d == 3 ? 5 : 3;
    const PassCfg *cf3[5] = {&p->cfg_xf, &p->cfg_yf, &p->cfg_conv, &p->cfg_yi, &p->cfg_xi};
    const PassCfg *cf2[3] = {&p->cfg_xf, &p->cfg_conv, &p->cfg_xi};
    for (int i = 0; i < hd.npasses; ++i) {
        const PassCfg *c = p->d == 3 ? cf3[i] : cf2[i];
        hd.nl[i] = c->nl;
        hd.emax[i] = c->emax;
    }
    hd.L = p->L;
    hd.eps = p->eps;
    hd.delta = p->opt.delta;
    hd.gs_err = p->gs_err;
    hd.c0 = p->c0;
    hd.c2 = p->c2;
    hd.beta = p->opt.beta;
    hd.mult_elems = p->mult_elems;
    for (int a = 0; a < p->d; ++a)
        for (int st = 0; st < kMaxStages; ++st) {
            hd.radix[0][a][st] = st < p->sched_f[a].nst ? p->sched_f[a].r[st] : 0;
            hd.radix[1][a][st] = st < p->sched_i[a].nst ? p->sched_i[a].r[st] : 0;
        }
    unsigned char *b = static_cast<unsigned char *>(buf);
    memcpy(b, &hd, sizeof(hd));
    size_t off = sizeof(hd);
    const size_t wb = sizeof(double) * p->nterms, kb = sizeof(double) * p->mult_elems;
    GSM_CUDA_TRY(cudaSetDevice(p->device));
    GSM_CUDA_TRY(cudaMemcpy(b + off, p->d_w, wb, cudaMemcpyDeviceToHost));
    off += wb;
    GSM_CUDA_TRY(cudaMemcpy(b + off, p->d_tau, wb, cudaMemcpyDeviceToHost));
    off += wb;
    GSM_CUDA_TRY(cudaMemcpy(b + off, p->d_khat, kb, cudaMemcpyDeviceToHost));
    off += kb;
    const uint64_t sum = fnv1a(b, off);
    memcpy(b + off, &sum, sizeof(sum));
    return GSM_OK;
}

gsm_status_t gsm_plan_load(gsm_plan_t *out, const void *buf, size_t bytes, int precision, void *cuda_stream)
{
    if (!out || !buf) {
        set_error("out or buf is NULL");
        return GSM_ERR_INVALID_ARG;
    }
    *out = nullptr;
    const unsigned char *b = static_cast<const unsigned char *>(buf);
    SaveHeader hd;
    if (bytes < sizeof(hd) + sizeof(uint64_t)) {
        set_error("saved plan: buffer too short");
        return GSM_ERR_INVALID_ARG;
    }
    memcpy(&hd, b, sizeof(hd));
    if (hd.magic != kSaveMagic || hd.version != kSaveVersion || hd.header_bytes != sizeof(SaveHeader)) {
        set_error("saved plan: not a plan of this format version");
        return GSM_ERR_INVALID_ARG;
    }
    if (hd.d < 2 || hd.d > 3 || hd.nterms < 1 || hd.nterms > kGsCap) {
        set_error("saved plan: header out of range");
        return GSM_ERR_INVALID_ARG;
    }
    uint64_t me = 1;
    for (int a = 0; a < hd.d; ++a) {
        if (hd.n[a] < kMinN || hd.n[a] > kMaxM) {
            set_error("saved plan: header out of range");
            return GSM_ERR_INVALID_ARG;
        }
        me *= (uint64_t)(hd.n[a] + 1);
    }
    const size_t need = sizeof(hd) + sizeof(double) * (2 * (size_t)hd.nterms + me) + sizeof(uint64_t);
    if (hd.mult_elems != me || bytes != need) {
        set_error("saved plan: size does not match its header");
        return GSM_ERR_INVALID_ARG;
    }
    uint64_t sum;
    memcpy(&sum, b + need - sizeof(sum), sizeof(sum));
    if (sum != fnv1a(b, need - sizeof(sum))) {
        set_error("saved plan: checksum mismatch (corrupted data)");
        return GSM_ERR_INVALID_ARG;
    }
    // copy the arrays out (the buffer need not be 8-byte aligned)
    std::vector<double> w(hd.nterms), tau(hd.nterms), khat(me);
    size_t off = sizeof(hd);
    memcpy(w.data(), b + off, sizeof(double) * hd.nterms);
    off += sizeof(double) * hd.nterms;
    memcpy(tau.data(), b + off, sizeof(double) * hd.nterms);
    off += sizeof(double) * hd.nterms;
    memcpy(khat.data(), b + off, sizeof(double) * me);

    gsm_options_t o;
    gsm_default_options(&o);
    o.delta = hd.delta;
    o.beta = hd.beta;
    o.S = hd.S;
    o.precision = (gsm_precision_t)(precision >= 0 ? precision : hd.precision);
    for (int a = 0; a < 3; ++a) {
        o.dip_n[a] = hd.dip_n[a];
        o.dip_m[a] = hd.dip_m[a];
    }
    StoredPlanData sd;
    sd.L = hd.L;
    for (int a = 0; a < 3; ++a) sd.eta[a] = hd.eta[a];
    sd.S = hd.S;
    sd.nterms = hd.nterms;
    sd.gs_err = hd.gs_err;
    sd.c0 = hd.c0;
    sd.c2 = hd.c2;
    sd.w = w.data();
    sd.tau = tau.data();
    sd.khat = khat.data();
    gsm_plan_t h = nullptr;
    gsm_status_t s = create_plan(&h, (gsm_kernel_t)hd.kind, hd.d, hd.L, hd.n, hd.eps, &o, cuda_stream, &sd);
    if (s != GSM_OK) return s;
    Plan *p = reinterpret_cast<Plan *>(h);
    p->eps = hd.eps;
    if (o.precision == hd.precision && hd.npasses == (hd.d == 3 ? 5 : 3)) {
        // the saved (possibly tuned) launch shapes; a shape this device
        // cannot run keeps the default
        for (int i = 0; i < hd.npasses; ++i)
            if (set_pass_shape(p, i, hd.nl[i], hd.emax[i]) != GSM_OK) set_error("");
        // and the saved schedules; a pair this plan cannot take keeps the default
        for (int a = 0; a < hd.d; ++a) {
            Sched sc[2];
            bool ok = true;
            for (int dir = 0; dir < 2 && ok; ++dir) {
                int r[kMaxStages], cnt = 0;
                while (cnt < kMaxStages && hd.radix[dir][a][cnt] != 0) {
                    r[cnt] = hd.radix[dir][a][cnt];
                    ++cnt;
                }
                ok = cnt > 0 && make_sched_order(p->M[a], r, cnt, dir == 0, &sc[dir]);
            }
            if (!ok || !axis_pair_ok(p, a, sc[0], sc[1])) continue;
            gsm_status_t ss = set_axis_pair(p, a, sc[0], sc[1], static_cast<cudaStream_t>(cuda_stream));
            if (ss == GSM_ERR_OOM) {
                release_handle(g_live_plans, p);
                free_plan(p);
                return ss;
            }
        }
    }
    *out = h;
    return GSM_OK;
}

gsm_status_t gsm_apply(gsm_plan_t h, const void *rho, void *u, void *cuda_stream)
{
    Plan *p = checked(h);
    if (!p) {
        set_error("bad plan handle");
        return GSM_ERR_BAD_PLAN;
    }
    if (!rho || !u) {
        set_error("rho or u is NULL");
        return GSM_ERR_INVALID_ARG;
    }
    return launch_apply(p, rho, u, static_cast<cudaStream_t>(cuda_stream));
}

gsm_status_t gsm_apply_pass(gsm_plan_t h, int pass, const void *rho, void *u, void *cuda_stream)
{
    Plan *p = checked(h);
    if (!p) {
        set_error("bad plan handle");
        return GSM_ERR_BAD_PLAN;
    }
    const int np = p->d == 3 ? 5 : 3;
    if (pass < 0 || pass >= np) {
        set_error("pass out of range");
        return GSM_ERR_INVALID_ARG;
    }
    if ((pass == 0 && !rho) || (pass == np - 1 && !u)) {
        set_error("rho or u is NULL");
        return GSM_ERR_INVALID_ARG;
    }
    return launch_pass(p, pass, rho, u, static_cast<cudaStream_t>(cuda_stream));
}

gsm_status_t gsm_plan_autotune(gsm_plan_t h, void *cuda_stream, char *report, size_t report_len)
{
    Plan *p = checked(h);
    if (!p) {
        set_error("bad plan handle");
        return GSM_ERR_BAD_PLAN;
    }
    std::string rep;
    gsm_status_t s = autotune_plan(p, static_cast<cudaStream_t>(cuda_stream), &rep);
    if (report && report_len > 0) {
        const size_t n = rep.size() < report_len - 1 ? rep.size() : report_len - 1;
        memcpy(report, rep.data(), n);
        report[n] = 0;
    }
    return s;
}

gsm_status_t gsm_apply_host(gsm_plan_t h, const void *rho_host, void *u_host, void *cuda_stream)
{
    Plan *p = checked(h);
    if (!p) {
        set_error("bad plan handle");
        return GSM_ERR_BAD_PLAN;
    }
    if (!rho_host || !u_host) {
        set_error("rho or u is NULL");
        return GSM_ERR_INVALID_ARG;
    }
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const size_t bytes = grid_points(p) * io_bytes(p);
    // Page-locked host arrays are mapped into the device's address space: the
    // x passes then read rho and write u in host memory themselves, over the
    // coherent host link, with no separate copies.  Anything else (pageable
    // memory) goes through the staging buffers below.
    cudaPointerAttributes ai, ao;
    const bool in_mapped = cudaPointerGetAttributes(&ai, rho_host) == cudaSuccess && ai.type == cudaMemoryTypeHost &&
                           ai.devicePointer != nullptr;
    const bool out_mapped = cudaPointerGetAttributes(&ao, u_host) == cudaSuccess && ao.type == cudaMemoryTypeHost &&
                            ao.devicePointer != nullptr;
    cudaGetLastError();   // an unregistered pointer may leave an error behind on older runtimes
    if (in_mapped && out_mapped && p->opt.host_zero_copy != 0) {
        gsm_status_t s = launch_apply(p, ai.devicePointer, ao.devicePointer, st);
        if (s != GSM_OK) return s;
        GSM_CUDA_TRY(cudaStreamSynchronize(st));
        return GSM_OK;
    }
    if (!p->d_stage_in || !p->d_stage_out) {
        // both buffers or neither: the plan keeps them only when both exist
        void *a = nullptr, *b = nullptr;
        cudaError_t e = dev_alloc(&a, bytes);
        if (e == cudaSuccess) e = dev_alloc(&b, bytes);
        if (e != cudaSuccess) {
            dev_free(a);
            dev_free(b);
            cudaGetLastError();
            set_error(std::string("host apply staging buffers: ") + cudaGetErrorString(e));
            return e == cudaErrorMemoryAllocation ? GSM_ERR_OOM : GSM_ERR_CUDA;
        }
        dev_free(p->d_stage_in);
        dev_free(p->d_stage_out);
        p->d_stage_in = a;
        p->d_stage_out = b;
    }
    if (p->d != 3) {
        GSM_CUDA_TRY(cudaMemcpyAsync(p->d_stage_in, rho_host, bytes, cudaMemcpyHostToDevice, st));
        gsm_status_t s = launch_apply(p, p->d_stage_in, p->d_stage_out, st);
        if (s != GSM_OK) return s;
        GSM_CUDA_TRY(cudaMemcpyAsync(u_host, p->d_stage_out, bytes, cudaMemcpyDeviceToHost, st));
        GSM_CUDA_TRY(cudaStreamSynchronize(st));
        return GSM_OK;
    }
    // 3D: the x passes work slab by slab, so the host-to-device copy of z-chunk c
    // overlaps the x forward pass of chunk c - 1, and the device-to-host copy of
    // chunk c the x inverse pass of chunk c + 1 (copies on the plan's own stream,
    // ordered against `st` by events)
    if (!p->copy_stream) {
        // the stream and all its events, or nothing
        cudaStream_t cs_new = nullptr;
        cudaEvent_t ev_new[2 * kHostChunks + 2] = {};
        cudaError_t e = cudaStreamCreateWithFlags(&cs_new, cudaStreamNonBlocking);
        for (cudaEvent_t &ev : ev_new)
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e != cudaSuccess) {
            for (cudaEvent_t ev : ev_new)
                if (ev) cudaEventDestroy(ev);
            if (cs_new) cudaStreamDestroy(cs_new);
            set_error(std::string("host apply copy stream: ") + cudaGetErrorString(e));
            return e == cudaErrorMemoryAllocation ? GSM_ERR_OOM : GSM_ERR_CUDA;
        }
        p->copy_stream = cs_new;
        for (int i = 0; i < 2 * kHostChunks + 2; ++i) p->copy_ev[i] = ev_new[i];
    }
    cudaStream_t cs = p->copy_stream;
    const int nz = p->n[2];
    const int K = nz < kHostChunks ? nz : kHostChunks;
    const size_t slab = (size_t)p->n[0] * p->n[1] * io_bytes(p);
    const unsigned char *hin = static_cast<const unsigned char *>(rho_host);
    unsigned char *hout = static_cast<unsigned char *>(u_host);
    unsigned char *din = static_cast<unsigned char *>(p->d_stage_in);
    unsigned char *dout = static_cast<unsigned char *>(p->d_stage_out);
    cudaEvent_t *ev_in = p->copy_ev, *ev_out = p->copy_ev + kHostChunks, ev_start = p->copy_ev[2 * kHostChunks],
                ev_done = p->copy_ev[2 * kHostChunks + 1];
    GSM_CUDA_TRY(cudaEventRecord(ev_start, st));          // work queued before on `st` comes first
    GSM_CUDA_TRY(cudaStreamWaitEvent(cs, ev_start, 0));
    for (int c = 0; c < K; ++c) {
        const int z0 = (int)((long)nz * c / K), z1 = (int)((long)nz * (c + 1) / K);
        GSM_CUDA_TRY(cudaMemcpyAsync(din + z0 * slab, hin + z0 * slab, (z1 - z0) * slab, cudaMemcpyHostToDevice, cs));
        GSM_CUDA_TRY(cudaEventRecord(ev_in[c], cs));
        GSM_CUDA_TRY(cudaStreamWaitEvent(st, ev_in[c], 0));
        gsm_status_t s = launch_x_slabs(p, false, z0, z1, din, nullptr, st);
        if (s != GSM_OK) return s;
    }
    for (int pass = 1; pass <= 3; ++pass) {
        gsm_status_t s = launch_pass(p, pass, nullptr, nullptr, st);
        if (s != GSM_OK) return s;
    }
    for (int c = 0; c < K; ++c) {
        const int z0 = (int)((long)nz * c / K), z1 = (int)((long)nz * (c + 1) / K);
        gsm_status_t s = launch_x_slabs(p, true, z0, z1, nullptr, dout, st);
        if (s != GSM_OK) return s;
        GSM_CUDA_TRY(cudaEventRecord(ev_out[c], st));
        GSM_CUDA_TRY(cudaStreamWaitEvent(cs, ev_out[c], 0));
        GSM_CUDA_TRY(cudaMemcpyAsync(hout + z0 * slab, dout + z0 * slab, (z1 - z0) * slab, cudaMemcpyDeviceToHost, cs));
    }
    GSM_CUDA_TRY(cudaEventRecord(ev_done, cs));
    GSM_CUDA_TRY(cudaStreamWaitEvent(st, ev_done, 0));     // later work on `st` sees u
    GSM_CUDA_TRY(cudaStreamSynchronize(st));
    return GSM_OK;
}

static gsm_status_t check_batch_args(int count, const gsm_plan_t *plans, const void *const *rho, void *const *u,
                                     std::vector<const Plan *> *out)
{
    if (count < 0 || (count > 0 && (!plans || !rho || !u))) {
        set_error("bad batch arguments");
        return GSM_ERR_INVALID_ARG;
    }
    for (int i = 0; i < count; ++i) {
        const Plan *p = checked(plans[i]);
        if (!p) {
            set_error("bad plan handle in batch");
            return GSM_ERR_BAD_PLAN;
        }
        if (!rho[i] || !u[i]) {
            set_error("NULL array in batch");
            return GSM_ERR_INVALID_ARG;
        }
        for (int j = 0; j < i; ++j)
            if (plans[j] == plans[i]) {
                set_error("a plan appears twice in one batch (its workspace is shared)");
                return GSM_ERR_INVALID_ARG;
            }
        out->push_back(p);
    }
    return GSM_OK;
}

gsm_status_t gsm_apply_batched(int count, const gsm_plan_t *plans, const void *const *rho, void *const *u,
                               void *cuda_stream)
{
    std::vector<const Plan *> ps;
    gsm_status_t s = check_batch_args(count, plans, rho, u, &ps);
    if (s != GSM_OK || count == 0) return s;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    void *state = nullptr;
    GSM_CUDA_TRY(dev_alloc_async_bytes(&state, batch_state_bytes(count), st));
    s = launch_batched(count, ps.data(), rho, u, kBatchLines, st, false, static_cast<unsigned *>(state));
    if (s != GSM_OK) {
        dev_free_async(state, st);
        return s;
    }
    s = batch_status(static_cast<const unsigned *>(state), count, st);
    dev_free_async(state, st);
    return s;
}

}  // extern "C"

namespace gsm {
constexpr uint64_t kBatchMagic = 0x47534d4241544348ull;   // "GSMBATCH"
struct Batch {
    uint64_t magic = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int count = 0;
    int nl = 0;               // lines (warps) per CTA chosen by timing
    unsigned *state = nullptr;   // work-queue state of the recorded launches
};
}  // namespace gsm

extern "C" {

gsm_status_t gsm_batch_create(gsm_batch_t *out, int count, const gsm_plan_t *plans, const void *const *rho,
                              void *const *u, void *cuda_stream)
{
    if (!out) {
        set_error("out is NULL");
        return GSM_ERR_INVALID_ARG;
    }
    *out = nullptr;
    std::vector<const Plan *> ps;
    gsm_status_t s = check_batch_args(count, plans, rho, u, &ps);
    if (s != GSM_OK) return s;
    if (count == 0) {
        set_error("empty batch");
        return GSM_ERR_INVALID_ARG;
    }
    // kernels are prepared outside the capture, and the lines per CTA of the
    // grouped launches (4 or 8 warps) are chosen by timing both on the stream
    cudaStream_t ts = static_cast<cudaStream_t>(cuda_stream);
    unsigned *state = nullptr;
    GSM_CUDA_TRY(dev_alloc(&state, batch_state_bytes(count)));
    int best_nl = kBatchLines;
    {
        float best_ms = 1e30f;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        cudaError_t ec = cudaEventCreate(&e0);
        if (ec == cudaSuccess) ec = cudaEventCreate(&e1);
        if (ec != cudaSuccess) {
            if (e0) cudaEventDestroy(e0);
            dev_free(state);
            GSM_CUDA_TRY(ec);
        }
        for (int nl : {4, 8}) {
            s = launch_batched(count, ps.data(), rho, u, nl, ts, true, state);
            if (s == GSM_OK) s = launch_batched(count, ps.data(), rho, u, nl, ts, false, state);
            cudaEventRecord(e0, ts);
            if (s == GSM_OK) s = launch_batched(count, ps.data(), rho, u, nl, ts, false, state);
            cudaEventRecord(e1, ts);
            cudaError_t e = cudaEventSynchronize(e1);
            if (s == GSM_OK && e == cudaSuccess) s = batch_status(state, count, ts);
            if (s != GSM_OK || e != cudaSuccess) {
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                dev_free(state);
                if (s == GSM_OK) {
                    set_error(std::string("batch timing: ") + cudaGetErrorString(e));
                    s = GSM_ERR_CUDA;
                }
                return s;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best_ms) {
                best_ms = ms;
                best_nl = nl;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    }
    cudaStream_t cs;
    cudaError_t ecs = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (ecs != cudaSuccess) {
        dev_free(state);
        GSM_CUDA_TRY(ecs);
    }
    Batch *b = new (std::nothrow) Batch();
    if (!b) {
        cudaStreamDestroy(cs);
        dev_free(state);
        set_error("host allocation failed");
        return GSM_ERR_OOM;
    }
    b->state = state;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        s = launch_batched(count, ps.data(), rho, u, best_nl, cs, false, state);
        cudaGraph_t g = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(cs, &g);
        if (s == GSM_OK && e2 != cudaSuccess) e = e2;
        b->graph = g;
        if (s == GSM_OK && e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, g, 0);
    }
    cudaStreamDestroy(cs);
    if (s == GSM_OK && e != cudaSuccess) {
        set_error(std::string("batch graph: ") + cudaGetErrorString(e));
        s = e == cudaErrorMemoryAllocation ? GSM_ERR_OOM : GSM_ERR_CUDA;
    }
    if (s != GSM_OK) {
        if (b->exec) cudaGraphExecDestroy(b->exec);
        if (b->graph) cudaGraphDestroy(b->graph);
        dev_free(b->state);
        delete b;
        return s;
    }
    b->count = count;
    b->nl = best_nl;
    b->magic = kBatchMagic;
    register_handle(g_live_batches, b);
    *out = reinterpret_cast<gsm_batch_t>(b);
    return GSM_OK;
}

static Batch *checked_batch(gsm_batch_t h)
{
    if (!is_live(g_live_batches, h)) return nullptr;
    Batch *b = reinterpret_cast<Batch *>(h);
    return b->magic == kBatchMagic ? b : nullptr;
}

gsm_status_t gsm_batch_launch(gsm_batch_t h, void *cuda_stream)
{
    Batch *b = checked_batch(h);
    if (!b) {
        set_error("bad batch handle");
        return GSM_ERR_BAD_PLAN;
    }
    GSM_CUDA_TRY(cudaGraphLaunch(b->exec, static_cast<cudaStream_t>(cuda_stream)));
    return GSM_OK;
}

gsm_status_t gsm_batch_wait(gsm_batch_t h, void *cuda_stream)
{
    Batch *b = checked_batch(h);
    if (!b) {
        set_error("bad batch handle");
        return GSM_ERR_BAD_PLAN;
    }
    return batch_status(b->state, b->count, static_cast<cudaStream_t>(cuda_stream));
}

gsm_status_t gsm_batch_destroy(gsm_batch_t h)
{
    Batch *b = checked_batch(h);
    if (!b) {
        set_error("bad batch handle");
        return GSM_ERR_BAD_PLAN;
    }
    release_handle(g_live_batches, b);
    cudaDeviceSynchronize();
    cudaGraphExecDestroy(b->exec);
    cudaGraphDestroy(b->graph);
    dev_free(b->state);
    b->magic = 0;
    delete b;
    return GSM_OK;
}

gsm_status_t gsm_hartree(gsm_plan_t h, const void *psi, void *u, void *energy, void *grad, void *cuda_stream)
{
    Plan *p = checked(h);
    if (!p) {
        set_error("bad plan handle");
        return GSM_ERR_BAD_PLAN;
    }
    if (!psi || !u || !energy) {
        set_error("psi, u or energy is NULL");
        return GSM_ERR_INVALID_ARG;
    }
    return launch_hartree(p, psi, u, energy, grad, static_cast<cudaStream_t>(cuda_stream));
}

gsm_status_t gsm_plan_info(gsm_plan_t h, gsm_plan_info_t *info)
{
    Plan *p = checked(h);
    if (!p) {
        set_error("bad plan handle");
        return GSM_ERR_BAD_PLAN;
    }
    if (!info) {
        set_error("info is NULL");
        return GSM_ERR_INVALID_ARG;
    }
    memset(info, 0, sizeof(*info));
    info->kernel = p->kind;
    info->d = p->d;
    for (int a = 0; a < 3; ++a) {
        info->n[a] = a < p->d ? p->n[a] : 1;
        info->M[a] = a < p->d ? p->M[a] : 1;
    }
    info->L = p->L;
    for (int a = 0; a < p->d; ++a) info->box[a] = p->L * p->eta[a];
    info->beta = p->opt.beta;
    info->delta = p->opt.delta;
    info->S = p->S;
    info->nterms = p->nterms;
    info->gs_err = p->gs_err;
    info->c0 = p->c0;
    info->c2 = p->c2;
    info->precision = p->opt.precision;
    const size_t me = p->opt.precision == GSM_FP64 ? 8 : (p->opt.precision == GSM_FP32 ? 4 : 8);
    info->bytes_multiplier = p->mult_elems_pass * me;
    info->bytes_workspace = p->work1_bytes + p->work2_bytes;
    info->npasses = p->d == 3 ? 5 : 3;
    const PassCfg *cf3[5] = {&p->cfg_xf, &p->cfg_yf, &p->cfg_conv, &p->cfg_yi, &p->cfg_xi};
    const PassCfg *cf2[3] = {&p->cfg_xf, &p->cfg_conv, &p->cfg_xi};
    for (int i = 0; i < info->npasses; ++i) {
        const PassCfg *c = p->d == 3 ? cf3[i] : cf2[i];
        info->launch_nl[i] = c->nl;
        info->launch_threads[i] = c->gthr;
        info->launch_emax[i] = c->emax;
    }
    for (int a = 0; a < p->d; ++a)
        for (int st = 0; st < 12 && st < kMaxStages; ++st) {
            info->radix_fwd[a][st] = st < p->sched_f[a].nst ? p->sched_f[a].r[st] : 0;
            info->radix_inv[a][st] = st < p->sched_i[a].nst ? p->sched_i[a].r[st] : 0;
        }
    return GSM_OK;
}

gsm_status_t gsm_plan_set_schedule(gsm_plan_t h, int axis, int inverse, const int *radices, int count,
                                   void *cuda_stream)
{
    Plan *p = checked(h);
    if (!p) {
        set_error("bad plan handle");
        return GSM_ERR_BAD_PLAN;
    }
    if (axis < 0 || axis >= p->d || !radices) {
        set_error("axis out of range or radices NULL");
        return GSM_ERR_INVALID_ARG;
    }
    Sched sc;
    if (!make_sched_order(p->M[axis], radices, count, inverse == 0, &sc)) {
        set_error("radices must be 8, 4, 2, 5 or 3 with product 2n of the axis (forward: even first radix)");
        return GSM_ERR_INVALID_ARG;
    }
    return set_axis_schedule(p, axis, inverse != 0, sc, static_cast<cudaStream_t>(cuda_stream));
}

gsm_status_t gsm_plan_destroy(gsm_plan_t h)
{
    Plan *p = checked(h);
    if (!p) {
        set_error("bad plan handle");
        return GSM_ERR_BAD_PLAN;
    }
    release_handle(g_live_plans, p);
    cudaDeviceSynchronize();
    free_plan(p);
    return GSM_OK;
}

gsm_status_t gsm_plan_gs_terms(gsm_plan_t h, double *w_host, double *tau_host, int cap, int *nterms)
{
    Plan *p = checked(h);
    if (!p) {
        set_error("bad plan handle");
        return GSM_ERR_BAD_PLAN;
    }
    if (!w_host || !tau_host || !nterms || cap < 0) {
        set_error("NULL output");
        return GSM_ERR_INVALID_ARG;
    }
    *nterms = p->nterms;
    const int c = cap < p->nterms ? cap : p->nterms;
    GSM_CUDA_TRY(cudaMemcpy(w_host, p->d_w, sizeof(double) * c, cudaMemcpyDeviceToHost));
    GSM_CUDA_TRY(cudaMemcpy(tau_host, p->d_tau, sizeof(double) * c, cudaMemcpyDeviceToHost));
    return GSM_OK;
}

gsm_status_t gsm_plan_kernel_tensor(gsm_plan_t h, double *host_out, size_t count)
{
    Plan *p = checked(h);
    if (!p) {
        set_error("bad plan handle");
        return GSM_ERR_BAD_PLAN;
    }
    if (!host_out || count != p->mult_elems) {
        set_error("output NULL or count does not match prod(n + 1)");
        return GSM_ERR_INVALID_ARG;
    }
    GSM_CUDA_TRY(cudaMemcpy(host_out, p->d_khat, sizeof(double) * count, cudaMemcpyDeviceToHost));
    return GSM_OK;
}

gsm_status_t gsm_plan_factors(gsm_plan_t h, int axis, double *host_out, size_t count)
{
    Plan *p = checked(h);
    if (!p) {
        set_error("bad plan handle");
        return GSM_ERR_BAD_PLAN;
    }
    if (axis < 0 || axis >= p->d || !host_out || count != (size_t)p->nterms * (p->n[axis] + 1)) {
        set_error("bad axis, NULL output or count != nterms * (n + 1)");
        return GSM_ERR_INVALID_ARG;
    }
    GSM_CUDA_TRY(cudaMemcpy(host_out, p->d_g[axis], sizeof(double) * count, cudaMemcpyDeviceToHost));
    return GSM_OK;
}

gsm_status_t gsm_fft_lines(int M, int nlines, int sign, gsm_precision_t precision, const double *in_dev,
                           double *out_dev, void *cuda_stream)
{
    if (!in_dev || !out_dev || nlines < 0 || (sign != 1 && sign != -1) || precision < GSM_FP64 ||
        precision > GSM_FP32X2) {
        set_error("bad FFT arguments");
        return GSM_ERR_INVALID_ARG;
    }
    if (nlines == 0) return GSM_OK;
    return launch_fft_lines(M, nlines, sign, precision, in_dev, out_dev, static_cast<cudaStream_t>(cuda_stream));
}

gsm_status_t gsm_fft_lines_noalloc(int M, int nlines, int sign, gsm_precision_t precision, const double *in_dev,
                                   double *out_dev, void *cuda_stream)
{
    if (!in_dev || !out_dev || nlines < 0 || (sign != 1 && sign != -1) || precision < GSM_FP64 ||
        precision > GSM_FP32X2) {
        set_error("bad FFT arguments");
        return GSM_ERR_INVALID_ARG;
    }
    if (nlines == 0) return GSM_OK;
    return launch_fft_lines_noalloc(M, nlines, sign, precision, in_dev, out_dev,
                                    static_cast<cudaStream_t>(cuda_stream));
}

gsm_status_t gsm_dft32_tc(int nvec, int sign, const double *in_dev, double *out_dev, void *cuda_stream)
{
    if (!in_dev || !out_dev || nvec < 0 || (sign != 1 && sign != -1)) {
        set_error("bad DFT arguments");
        return GSM_ERR_INVALID_ARG;
    }
    if (nvec == 0) return GSM_OK;
    return launch_dft32_tc(nvec, sign, in_dev, out_dev, static_cast<cudaStream_t>(cuda_stream));
}

gsm_status_t gsm_debug_fail_alloc(int k)
{
    g_fail_in.store(k < 0 ? -1 : (long)k);
    return GSM_OK;
}

gsm_status_t gsm_debug_batch_wait(long long wait_ns, int hold_instance)
{
    set_batch_wait(wait_ns > 0 ? (unsigned long long)wait_ns : 0ull, hold_instance);
    return GSM_OK;
}

gsm_status_t gsm_debug_alloc_stats(size_t *count, size_t *bytes)
{
    if (!count || !bytes) {
        set_error("count or bytes is NULL");
        return GSM_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lock(g_alloc_mutex);
    *count = g_alloc_live.size();
    *bytes = g_alloc_bytes;
    return GSM_OK;
}

}  // extern "C"
