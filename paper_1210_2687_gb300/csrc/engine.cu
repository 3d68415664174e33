// engine.cu -- host engine and C ABI of the batched mask-decoupled ADMM.
//
// A plan owns one problem's device state (the duals d1, d2, the two
// half-spectrum buffers exchanged between the row and column phases, the
// spectra Lambda and K, M^T y and the effective mask). admm_deconv_solve_batch
// groups problems of equal (H, W, regulariser) and advances each group with
// one column-phase and one row-phase launch per iteration; a device control
// block per problem counts iterations and retires the problem when its stop
// rule holds (Sec. V: relative change of the objective; or of x; or a fixed
// iteration count). The host polls the number of active problems once per
// chunk of iterations, one chunk behind the device.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>

#include "../../include/admm_deconv.h"
#include "kernels.cuh"
#include "haar.cuh"
#include "cg.cuh"
#include "gen.cuh"
#include "setup.cuh"
#include "variants.cuh"

using namespace admm;

namespace admm {
// the learned warm start of admm_warmstart_load (cnn.cu)
bool ws_loaded();
int ws_batch_limit(int H, int W);
int ws_predict_starts(int count, int H, int W, const float* const* ybar, const uint8_t* const* mask,
                      float* const* x0, float* const* d0, cudaStream_t s);
// the driver's tensor-map encoder (cnn.cu)
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encode_fn();

// ADMM_OPT_FAIL_ALLOC: allocations left before the injected failure (0 = off)
static std::atomic<long long> g_fail_alloc{0};
bool alloc_fault_fire() {
    long long v = g_fail_alloc.load();
    while (v > 0) {
        if (g_fail_alloc.compare_exchange_weak(v, v - 1)) return v == 1;
    }
    return false;
}
}  // namespace admm

struct admm_plan_s {
    admm_params_t p{};
    std::vector<float> psf;
    std::vector<float> band_mu;  // one penalty per frame band (empty: mu2 for all)
    int device = 0;
    int Wc = 0, Wp = 0, cb = 0, R = 0, n_strips = 0, n_slots = 0, nb = 0, levels = 0;
    int row_v = 0, col_v = 0, slot_ctas = 0, lanes = 0;   // launch configuration (tuning table at plan time)
    int fam = ADMM_REG_TV;      // kernel family: ADMM_REG_TV (isotropic or anisotropic) or ADMM_REG_HAAR
    float lam = 0.f, mu1 = 0.f, mu2 = 0.f;
    void* slab = nullptr;
    float4* Sa = nullptr;
    float4* Sb = nullptr;
    float* d1 = nullptr;
    float* d2 = nullptr;
    float* ybar = nullptr;
    float* xprev = nullptr;
    float* work = nullptr;      // frame prior and Reeves-Sorel variants: x / zeta1 / w scratch planes
    float* cg = nullptr;        // Reeves-Sorel variants: x~, A x~, v, A v, s, z planes
    double* cg_part = nullptr;  // ... and the CG step's partial sums
    uint8_t* mask = nullptr;
    float2* lamT = nullptr;
    float* kT = nullptr;
    double* partials = nullptr;
    ProbCtl* ctl = nullptr;
    float* ystage = nullptr;
    uint8_t* mstage = nullptr;
    float* xstage = nullptr;
    float* psf_dev = nullptr;
    void* zmap = nullptr;        // frame prior: the synthesis tile's TMA tensor maps (levels + 1)
    uint32_t* zbits = nullptr;   // frame analysis prior: two bits per band and pixel (beside zeta2)
    int last_iter = 0;          // iterations of the last solve: d2 lives in buffer last_iter & 1
    int warm_mode = 0;          // the next solve starts from: 0 u0 = d0 = 0; 1 admm_deconv_warm_start's
                                // (x0, d0); 2 admm_deconv_set_state's state (resume)
    int Hu = 0, Wu = 0;         // the caller's image size (p.H x p.W is the domain solved on)
    bool padded = false;        // Hu x Wu sits in the top-left corner of a larger domain
    bool gen = false;           // a side is not a power of two: the mixed-radix kernels (gen.cuh)
};

namespace {

std::mutex g_mutex;

struct DeviceCtx {
    bool ready = false;
    float2* tw = nullptr;            // exp(-2 pi i k / 2048), k < 2048, then the per-pass tables
    ProbDesc* desc = nullptr;        // descriptor table
    float** xptr = nullptr;          // finalize destinations
    int cap = 0;
    int* n_active = nullptr;         // unretired problems per size class (cap entries)
    int* queue = nullptr;            // next problem of the pool to start
    int* slot_map = nullptr;         // problem index per launch slot (cap entries)
    int* h_active = nullptr;         // pinned, 2 x cap (double-buffered copy of n_active)
    ProbCtl* h_ctl = nullptr;        // pinned copy-back area
    ProbDesc* h_desc = nullptr;      // pinned staging for the table
    PrepItem* prep = nullptr;        // input preparation of a batch call (cap entries)
    PrepItem* h_prep = nullptr;      // ... pinned staging
    float** h_xptr = nullptr;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    static constexpr int kBranches = 8;             // capture streams (graph branches)
    cudaStream_t branch[kBranches] = {};
    cudaEvent_t fork_ev = nullptr;
    cudaEvent_t join_ev[kBranches] = {};
    // chunk graphs keyed by the batch's layout (size classes, offsets, slots,
    // lanes); cleared whenever the descriptor or slot tables move
    std::map<std::string, cudaGraphExec_t> graphs;
    // mixed-radix twiddles exp(-2 pi i k / N), k < N, per length N
    std::map<int, float2*> gtw;
};

// A group's problems split into `n` lanes that iterate independently: lane
// l owns problems [off[l], off[l] + cnt[l]) of the descriptor table and
// slots [soff[l], soff[l] + slots[l]). In a replayed chunk the lanes are
// independent graph branches, so one lane's column phase (transform-bound)
// can share the GPU with the other lane's row phase (memory-bound).
constexpr int kMaxLanes = 4;
constexpr int kDefaultLanes = 2;
struct Lanes {
    int n = 1;
    int off[kMaxLanes] = {}, cnt[kMaxLanes] = {}, soff[kMaxLanes] = {}, slots[kMaxLanes] = {};
};
std::map<int, DeviceCtx> g_ctx;

struct Profile {
    bool on = false;
    admm_profile_t acc{};
    std::vector<cudaEvent_t> ev;     // reused across solves
} g_prof;

long long g_launches = 0;            // every kernel launched (under g_mutex)
int g_max_slots = 0;                 // ADMM_OPT_MAX_SLOTS
int g_test_stall = 0;                // ADMM_OPT_TEST_STALL: armed for the next solve

int prof_event(size_t i, cudaStream_t s) {
    while (g_prof.ev.size() <= i) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return ADMM_ECUDA;
        g_prof.ev.push_back(e);
    }
    return cudaEventRecord(g_prof.ev[i], s) == cudaSuccess ? ADMM_OK : ADMM_ECUDA;
}

bool is_pow2_size(int n) { return n >= 64 && n <= 2048 && (n & (n - 1)) == 0; }

// smallest power-of-two transform size >= n (-1 if there is none)
int next_supported_size(int n) {
    if (n < 1 || n > 2048) return -1;
    int m = 64;
    while (m < n) m <<= 1;
    return m;
}
// sides of the mixed-radix path: m 2^k, m in {1, 3, 5}, multiples of 32, 64..2048
bool is_gen_size(int n) { return gfft_length_ok(n); }
// smallest side >= n the mixed-radix path takes (-1 if there is none)
int next_gen_size(int n) {
    for (int m = std::max(n, 64); m <= 2048; ++m)
        if (is_gen_size(m)) return m;
    return -1;
}

int cuda_fail(cudaError_t e) {
    return e == cudaErrorMemoryAllocation ? ADMM_ENOMEM : ADMM_ECUDA;
}
#define CK(call)                                   \
    do {                                           \
        cudaError_t e_ = (call);                   \
        if (e_ != cudaSuccess) return cuda_fail(e_); \
    } while (0)

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// device and pinned-host allocations of the library go through these, so
// that ADMM_OPT_FAIL_ALLOC can make one of them fail (host-side fault
// injection for the ADMM_ENOMEM paths)
cudaError_t dev_alloc(void** p, size_t bytes) {
    if (alloc_fault_fire()) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}
template <typename T> cudaError_t dev_alloc(T** p, size_t bytes) {
    void* v = nullptr;
    const cudaError_t e = dev_alloc(&v, bytes);
    *p = static_cast<T*>(v);
    return e;
}
template <typename T> cudaError_t host_alloc(T** p, size_t bytes) {
    if (alloc_fault_fire()) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    void* v = nullptr;
    const cudaError_t e = cudaHostAlloc(&v, bytes, cudaHostAllocDefault);
    *p = static_cast<T*>(v);
    return e;
}

int ensure_ctx(int dev, int count, DeviceCtx** out) {
    DeviceCtx& c = g_ctx[dev];
    if (!c.ready) {
        // each resource is created once; a failed attempt resumes where it stopped
        if (!c.tw) {
            // the 2048-entry table, then the per-pass tables of every length
            std::vector<float2> tw(kTwiddleEntries, make_float2(0.f, 0.f));
            for (int k = 0; k < 2048; ++k) {
                // exact reduction: angle = 2 pi k / 2048
                const double a = 2.0 * M_PI * (double)k / 2048.0;
                tw[k] = make_float2((float)std::cos(a), (float)(-std::sin(a)));
            }
            for (int lg = 6, slot = 1; lg <= 11; ++lg, ++slot)
                fill_pass_table(1 << lg, tw.data(), tw.data() + 2048 * slot);
            float2* t = nullptr;
            CK(dev_alloc(&t, kTwiddleEntries * sizeof(float2)));
            if (cudaMemcpy(t, tw.data(), kTwiddleEntries * sizeof(float2), cudaMemcpyHostToDevice) != cudaSuccess) {
                cudaFree(t);
                return ADMM_ECUDA;
            }
            c.tw = t;
        }
        for (int i = 0; i < 2; ++i)
            if (!c.ev[i]) CK(cudaEventCreateWithFlags(&c.ev[i], cudaEventDisableTiming));
        for (int b = 0; b < DeviceCtx::kBranches; ++b) {
            if (!c.branch[b]) CK(cudaStreamCreateWithFlags(&c.branch[b], cudaStreamNonBlocking));
            if (!c.join_ev[b]) CK(cudaEventCreateWithFlags(&c.join_ev[b], cudaEventDisableTiming));
        }
        if (!c.fork_ev) CK(cudaEventCreateWithFlags(&c.fork_ev, cudaEventDisableTiming));
        c.ready = true;
    }
    if (count > c.cap || !c.desc) {
        int cap = std::max(count, 2 * c.cap);
        for (auto& kv : c.graphs) cudaGraphExecDestroy(kv.second);
        c.graphs.clear();
        if (c.desc) cudaFree(c.desc);
        if (c.xptr) cudaFree(c.xptr);
        if (c.slot_map) cudaFree(c.slot_map);
        if (c.queue) cudaFree(c.queue);
        if (c.n_active) cudaFree(c.n_active);
        if (c.h_active) cudaFreeHost(c.h_active);
        if (c.h_ctl) cudaFreeHost(c.h_ctl);
        if (c.h_desc) cudaFreeHost(c.h_desc);
        if (c.h_xptr) cudaFreeHost(c.h_xptr);
        if (c.prep) cudaFree(c.prep);
        if (c.h_prep) cudaFreeHost(c.h_prep);
        c.desc = nullptr; c.xptr = nullptr; c.h_ctl = nullptr; c.h_desc = nullptr; c.h_xptr = nullptr;
        c.prep = nullptr; c.h_prep = nullptr;
        c.slot_map = nullptr;
        c.queue = nullptr;
        c.n_active = nullptr;
        c.h_active = nullptr;
        c.cap = 0;
        // (on a failure the pointers allocated so far stay set with cap = 0: the
        // next call frees them and tries again)
        CK(dev_alloc(&c.desc, cap * sizeof(ProbDesc)));
        CK(dev_alloc(&c.slot_map, cap * sizeof(int)));
        CK(dev_alloc(&c.queue, kMaxLanes * cap * sizeof(int)));   // one word per lane
        CK(dev_alloc(&c.xptr, cap * sizeof(float*)));
        CK(dev_alloc(&c.n_active, cap * sizeof(int)));
        CK(host_alloc(&c.h_active, 2 * cap * sizeof(int)));
        CK(host_alloc(&c.h_ctl, cap * sizeof(ProbCtl)));
        CK(host_alloc(&c.h_desc, cap * sizeof(ProbDesc)));
        CK(host_alloc(&c.h_xptr, cap * sizeof(float*)));
        CK(dev_alloc(&c.prep, cap * sizeof(PrepItem)));
        CK(host_alloc(&c.h_prep, cap * sizeof(PrepItem)));
        c.cap = cap;
    }
    *out = &c;
    return ADMM_OK;
}

// the mixed-radix twiddle table of length N on this context (made on first use)
int gen_twiddles(DeviceCtx* c, int N, const float2** out) {
    auto it = c->gtw.find(N);
    if (it != c->gtw.end()) {
        *out = it->second;
        return ADMM_OK;
    }
    std::vector<float2> tw(N);
    for (int k = 0; k < N; ++k) {
        // exact reduction: angle = 2 pi k / N
        const double a = 2.0 * M_PI * (double)k / (double)N;
        tw[k] = make_float2((float)std::cos(a), (float)(-std::sin(a)));
    }
    float2* t = nullptr;
    CK(dev_alloc(&t, (size_t)N * sizeof(float2)));
    if (cudaMemcpy(t, tw.data(), (size_t)N * sizeof(float2), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(t);
        return ADMM_ECUDA;
    }
    c->gtw[N] = t;
    *out = t;
    return ADMM_OK;
}

// ---- tiling choices -----------------------------------------------------
// Defaults are entry 0 of the compiled candidate lists (variants.cuh); the
// tuning table overrides them per (device, H, W, regulariser, levels).
constexpr int kDefaultSlotCtas = 2400;

int col_block(int H) {
    const ColVariant* v = nullptr;
    return col_variants(H, &v) > 0 ? v[0].CB : 0;
}
int row_strip_tv(int W) {
    const RowVariant* v = nullptr;
    return tv_row_variants(W, &v) > 0 ? v[0].R : 0;
}

// launch slots of a group: enough problems in flight that a row-side launch
// has about `slot_ctas` CTAs (default some eight waves of two CTAs per SM on
// 152 SMs)
int choose_slots(int H, int W, bool tv, int R, int slot_ctas, int count) {
    const int per = tv ? H / R : haar_num_tiles(H, W);
    const int target = slot_ctas > 0 ? slot_ctas : kDefaultSlotCtas;
    int want = (target + per - 1) / per;
    if (g_max_slots > 0) want = std::min(want, g_max_slots);
    return std::max(1, std::min(count, want));
}

using TuneKey = std::tuple<int, int, int, int, int>;   // device, H, W, reg, levels
std::map<TuneKey, admm_tuning_t> g_tuning;            // under g_mutex

// the configuration a new plan of this class gets (entry 0 when untuned)
admm_tuning_t lookup_tuning(int dev, int H, int W, int reg, int levels) {
    auto it = g_tuning.find(TuneKey(dev, H, W, reg, levels));
    if (it != g_tuning.end()) return it->second;
    admm_tuning_t t{};
    t.H = H;
    t.W = W;
    t.reg = reg;
    t.haar_levels = levels;
    return t;
}

// fill the descriptive fields of `t` from its indices; false if an index is
// out of range for the class
bool describe_tuning(admm_tuning_t* t) {
    const ColVariant* cv = nullptr;
    const int nc = col_variants(t->H, &cv);
    if (t->col_variant < 0 || t->col_variant >= nc) return false;
    t->col_block = cv[t->col_variant].CB;
    t->col_min_ctas = cv[t->col_variant].MB;
    t->col_persistent = cv[t->col_variant].persistent;
    if (t->reg == ADMM_REG_TV) {
        const RowVariant* rv = nullptr;
        const int nr = tv_row_variants(t->W, &rv);
        if (t->row_variant < 0 || t->row_variant >= nr) return false;
        t->rows_per_strip = rv[t->row_variant].R;
        t->walk_depth = rv[t->row_variant].D;
        t->row_threads = rv[t->row_variant].NT;
    } else {
        if (t->row_variant != 0) return false;
        t->rows_per_strip = haar_row_strip(t->W);
        t->walk_depth = 0;
        t->row_threads = kThreads;
    }
    if (t->slot_ctas < 0 || t->lanes < 0 || t->lanes > kMaxLanes) return false;
    return true;
}

// default-configuration launches (the scratch-free entry point uses these)
cudaError_t launch_col(int H, const ProbDesc* d, SlotTable sl, int count, int Wc, int Wp, const float2* tw,
                       cudaStream_t s) {
    const ColVariant* v = nullptr;
    if (col_variants(H, &v) == 0) return cudaErrorInvalidValue;
    return v[0].fn(d, sl, count, Wc, Wp, tw, s);
}

cudaError_t launch_row_tv(int W, const ProbDesc* d, SlotTable sl, int count, int H, int Wp, const float2* tw,
                          int* n_active, cudaStream_t s) {
    const RowVariant* v = nullptr;
    if (tv_row_variants(W, &v) == 0) return cudaErrorInvalidValue;
    return v[0].fn(d, sl, count, H, Wp, tw, n_active, s);
}

template <int W>
cudaError_t launch_fin_t(const ProbDesc* d, float* const* xo, int count, int H, int Wp, const float2* tw,
                         cudaStream_t s) {
    constexpr int FT = W / 8, G = kThreads / FT;
    const size_t smem = (size_t)(G * W + W) * sizeof(float2);
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(finalize_x<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    dim3 grid((H + G - 1) / G, count);
    finalize_x<W><<<grid, kThreads, smem, s>>>(d, xo, H, Wp, tw);
    return cudaGetLastError();
}

cudaError_t launch_warm_rows(int W, const float* x0, float4* Sb, int H, int Wp, const float2* tw, cudaStream_t s) {
    const int G = kThreads / (W / 8);
    const size_t smem = (size_t)(G * W + W) * sizeof(float2);
    const unsigned grid = (unsigned)((H + G - 1) / G);
    switch (W) {
        case 64: warm_rows<64><<<grid, kThreads, smem, s>>>(x0, Sb, H, Wp, tw); break;
        case 128: warm_rows<128><<<grid, kThreads, smem, s>>>(x0, Sb, H, Wp, tw); break;
        case 256: warm_rows<256><<<grid, kThreads, smem, s>>>(x0, Sb, H, Wp, tw); break;
        case 512: warm_rows<512><<<grid, kThreads, smem, s>>>(x0, Sb, H, Wp, tw); break;
        case 1024: warm_rows<1024><<<grid, kThreads, smem, s>>>(x0, Sb, H, Wp, tw); break;
        case 2048: warm_rows<2048><<<grid, kThreads, smem, s>>>(x0, Sb, H, Wp, tw); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_fin(int W, const ProbDesc* d, float* const* xo, int count, int H, int Wp, const float2* tw,
                       cudaStream_t s) {
    switch (W) {
        case 64: return launch_fin_t<64>(d, xo, count, H, Wp, tw, s);
        case 128: return launch_fin_t<128>(d, xo, count, H, Wp, tw, s);
        case 256: return launch_fin_t<256>(d, xo, count, H, Wp, tw, s);
        case 512: return launch_fin_t<512>(d, xo, count, H, Wp, tw, s);
        case 1024: return launch_fin_t<1024>(d, xo, count, H, Wp, tw, s);
        case 2048: return launch_fin_t<2048>(d, xo, count, H, Wp, tw, s);
    }
    return cudaErrorInvalidValue;
}

bool is_device_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

void free_plan(admm_plan_s* pl) {
    if (!pl) return;
    if (pl->slab) cudaFree(pl->slab);
    delete pl;
}

// kernel family of a regulariser: ADMM_REG_TV for the priors whose row side
// is the TV row phase (isotropic or anisotropic), ADMM_REG_HAAR for those
// whose row side is a chain of row and tile kernels (the frame priors and the
// Reeves-Sorel variants); the family picks the tuning entry
int reg_family(int reg) { return (reg == ADMM_REG_TV || reg == ADMM_REG_TV_ANISO) ? ADMM_REG_TV : ADMM_REG_HAAR; }
bool reg_known(int reg) {
    return reg == ADMM_REG_TV || reg == ADMM_REG_HAAR || reg == ADMM_REG_TV_ANISO || reg == ADMM_REG_HAAR_LL_FREE ||
           reg == ADMM_REG_HAAR_SYNTHESIS || reg == ADMM_REG_TV_CG || reg == ADMM_REG_HAAR_CG;
}
bool reg_cg(int reg) { return reg == ADMM_REG_TV_CG || reg == ADMM_REG_HAAR_CG; }
// the TV prior (its x-step denominator has the difference spectra)
bool reg_tv_prior(int reg) { return reg == ADMM_REG_TV || reg == ADMM_REG_TV_ANISO || reg == ADMM_REG_TV_CG; }

ProbDesc make_desc(const admm_plan_s* pl) {
    ProbDesc d{};
    d.Sa = pl->Sa;
    d.Sb = pl->Sb;
    d.d1 = pl->d1;
    d.d2 = pl->d2;
    d.d2_stride = (long long)pl->nb * pl->p.H * pl->p.W;
    d.ybar = pl->ybar;
    d.mask = pl->mask;
    d.lamT = pl->lamT;
    d.kT = pl->kT;
    d.xprev = pl->xprev;
    d.work = pl->work;
    d.cg = pl->cg;
    d.cg_part = pl->cg_part;
    d.partials = pl->partials;
    d.ctl = pl->ctl;
    d.lam = pl->lam;
    d.mu1 = pl->mu1;
    d.mu2 = pl->mu2;
    d.gamma = (float)((double)pl->mu2 / (double)pl->mu1);
    d.tau = (float)((double)pl->lam / (double)pl->mu2);
    d.inv1pmu1 = (float)(1.0 / (1.0 + (double)pl->mu1));
    d.stop = pl->p.stop;
    d.max_iters = pl->p.max_iters;
    d.check_every = pl->p.check_every;
    d.n_strips = pl->n_strips;
    d.n_slots = pl->n_slots;
    d.warm = pl->warm_mode;
    d.test_stall = g_test_stall;
    d.zmap = pl->zmap;
    d.zbits = pl->zbits;
    d.ll_free = pl->p.reg == ADMM_REG_HAAR_LL_FREE ? 1 : 0;
    d.tol = pl->p.tol;
    for (int b = 0; b < 13; ++b) {
        const bool per = b < (int)pl->band_mu.size();
        d.band_tau[b] = per ? (float)((double)pl->lam / (double)pl->band_mu[b]) : d.tau;
        d.band_zs[b] = per ? (float)((double)pl->band_mu[b] / (double)pl->mu2) : 1.0f;
        d.band_izs[b] = per ? (float)((double)pl->mu2 / (double)pl->band_mu[b]) : 1.0f;
    }
    return d;
}

}  // namespace

// ===========================================================================
extern "C" {

const char* admm_deconv_version(void) { return "admm_deconv 0.1 (sm_103a)"; }

const char* admm_strerror(int code) {
    switch (code) {
        case ADMM_OK: return "ok";
        case ADMM_EINVAL: return "invalid argument";
        case ADMM_ENOMEM: return "out of memory";
        case ADMM_ECUDA: return "CUDA runtime error";
        case ADMM_EUNSUPPORTED_SIZE: return "unsupported image size (powers of two 64..2048)";
        case ADMM_ENONFINITE: return "iterate became non-finite";
        case ADMM_ETIMEOUT: return "device wait timed out";
    }
    return "unknown status";
}

int admm_deconv_plan(admm_plan_t* out, const admm_params_t* p, void* stream) {
    if (!out || !p || !p->psf) return ADMM_EINVAL;
    if (p->fft_pad_policy != ADMM_PAD_EXACT && p->fft_pad_policy != ADMM_PAD_NEXT) return ADMM_EINVAL;
    // the domain solved on: the caller's, or the next supported size (the
    // added rows and columns are more unknown boundary, Sec. IV-A)
    // Sides that are powers of two take the tuned power-of-two kernels; other
    // sides m 2^k (m = 3, 5) the mixed-radix kernels on the exact domain
    // (the Reeves-Sorel variants have no mixed-radix form and pad).
    int Hd = p->H, Wd = p->W;
    bool gen = false;
    if (!is_pow2_size(Hd) || !is_pow2_size(Wd)) {
        const bool gen_reg = !reg_cg(p->reg);
        if (gen_reg && is_gen_size(Hd) && is_gen_size(Wd)) {
            gen = true;
        } else if (p->fft_pad_policy == ADMM_PAD_NEXT) {
            Hd = gen_reg ? next_gen_size(p->H) : next_supported_size(p->H);
            Wd = gen_reg ? next_gen_size(p->W) : next_supported_size(p->W);
            if (Hd < 0 || Wd < 0) return ADMM_EUNSUPPORTED_SIZE;
            gen = !is_pow2_size(Hd) || !is_pow2_size(Wd);
        } else {
            return ADMM_EUNSUPPORTED_SIZE;
        }
    }
    if (p->psf_h < 1 || p->psf_w < 1 || (p->psf_h & 1) == 0 || (p->psf_w & 1) == 0) return ADMM_EINVAL;
    if (p->psf_h > std::min(p->H, kMaxPsfSide) || p->psf_w > std::min(p->W, kMaxPsfSide)) return ADMM_EINVAL;
    if (!(p->lambda >= 0.f) || !std::isfinite(p->lambda)) return ADMM_EINVAL;
    if (!reg_known(p->reg)) return ADMM_EINVAL;
    if (p->stop < ADMM_STOP_ITERS || p->stop > ADMM_STOP_REL_OBJ) return ADMM_EINVAL;
    if (p->max_iters <= 0 || p->check_every < 1 || !(p->tol >= 0.0)) return ADMM_EINVAL;
    const int fam = reg_family(p->reg);
    const bool cg = reg_cg(p->reg), tvp = reg_tv_prior(p->reg);
    const int levels = tvp ? 0 : (p->haar_levels == 0 ? 4 : p->haar_levels);
    if (!tvp && (levels < 1 || levels > kMaxHaarLevels)) return ADMM_EINVAL;
    double psum = 0.0;
    for (int i = 0; i < p->psf_h * p->psf_w; ++i) {
        if (!std::isfinite(p->psf[i])) return ADMM_EINVAL;
        psum += p->psf[i];
    }
    if (psum == 0.0) return ADMM_EINVAL;
    float mu1 = p->mu1, mu2 = p->mu2;
    if (mu2 <= 0.f) mu2 = 10.f * p->lambda;
    if (mu1 <= 0.f) mu1 = std::min(1.f, 3.f * mu2);
    if (!(mu1 > 0.f) || !(mu2 > 0.f)) return ADMM_EINVAL;
    // one penalty per frame band (eq. diagonal_penalty): FA-MD and its
    // low-low-free variant only
    if (p->band_mu) {
        if (p->reg != ADMM_REG_HAAR && p->reg != ADMM_REG_HAAR_LL_FREE) return ADMM_EINVAL;
        for (int b = 0; b < 3 * levels + 1; ++b)
            if (!(p->band_mu[b] > 0.f) || !std::isfinite(p->band_mu[b])) return ADMM_EINVAL;
    }

    std::lock_guard<std::mutex> lk(g_mutex);
    admm_plan_s* pl = new (std::nothrow) admm_plan_s();
    if (!pl) return ADMM_ENOMEM;
    pl->p = *p;
    pl->p.psf = nullptr;
    pl->p.band_mu = nullptr;
    if (p->band_mu) pl->band_mu.assign(p->band_mu, p->band_mu + 3 * levels + 1);
    pl->Hu = p->H;
    pl->Wu = p->W;
    pl->p.H = Hd;
    pl->p.W = Wd;
    pl->padded = Hd != p->H || Wd != p->W;
    pl->gen = gen;
    pl->psf.assign(p->psf, p->psf + p->psf_h * p->psf_w);
    pl->lam = p->lambda;
    pl->mu1 = mu1;
    pl->mu2 = mu2;
    pl->levels = levels;
    if (cudaGetDevice(&pl->device) != cudaSuccess) { free_plan(pl); return ADMM_ECUDA; }
    const int H = Hd, W = Wd;
    const size_t n = (size_t)H * W;
    pl->Wc = W / 2 + 1;
    if (gen) {
        // one configuration (no tuning); the row side is a kernel chain
        pl->cb = gen_col_block(H);
    } else {
        const admm_tuning_t tu = lookup_tuning(pl->device, H, W, fam, levels);
        const ColVariant* cv = nullptr;
        col_variants(H, &cv);
        pl->col_v = tu.col_variant;
        pl->row_v = tu.row_variant;
        pl->slot_ctas = tu.slot_ctas;
        pl->lanes = tu.lanes;
        pl->cb = cv[pl->col_v].CB;
    }
    pl->Wp = (int)align_up(pl->Wc, pl->cb);
    pl->fam = gen ? ADMM_REG_HAAR : fam;
    if (gen) {
        pl->R = gen_rows_per_cta(W);
        pl->nb = tvp ? 2 : 3 * levels + 1;
        pl->n_strips = tvp ? cg_num_tiles(H, W) : haar_num_tiles(H, W);
        pl->n_slots = H / pl->R + pl->n_strips;
    } else if (fam == ADMM_REG_TV) {
        const RowVariant* rv = nullptr;
        tv_row_variants(W, &rv);
        pl->R = rv[pl->row_v].R;
        pl->nb = 2;
    } else {
        pl->R = haar_row_strip(W);
        pl->nb = tvp ? 2 : 3 * levels + 1;
    }
    if (gen) {
    } else if (fam == ADMM_REG_TV) {
        pl->n_strips = H / pl->R;
        pl->n_slots = pl->n_strips;
    } else {
        // the tile kernel finishes the iteration; it also sums the row kernels' partials
        pl->n_strips = cg && tvp ? cg_num_tiles(H, W) : haar_num_tiles(H, W);
        pl->n_slots = haar_num_row_ctas(H, W) + pl->n_strips;
    }

    // one slab for everything the plan owns
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes, 256); return o; };
    const size_t oSa = take((size_t)H * pl->Wp * sizeof(float4));
    const size_t oSb = take((size_t)H * pl->Wp * sizeof(float4));
    const size_t od1 = take(n * sizeof(float));
    const size_t od2 = take(2 * (size_t)pl->nb * n * sizeof(float));
    const size_t oyb = take(n * sizeof(float));
    const size_t oxp = take(n * sizeof(float));
    const size_t owk = take(pl->fam == ADMM_REG_HAAR ? 3 * n * sizeof(float) : 0);
    const size_t ocg = take(cg ? 6 * n * sizeof(float) : 0);
    const size_t ocp = take(cg ? 2 * (size_t)haar_num_row_ctas(H, W) * sizeof(double) : 0);
    const size_t omk = take(n);
    const size_t olm = take((size_t)pl->Wc * H * sizeof(float2));
    const size_t okt = take((size_t)pl->Wc * H * sizeof(float));
    const size_t opt = take((size_t)pl->n_slots * kNumPartials * sizeof(double));
    const size_t oct = take(sizeof(ProbCtl));
    const size_t oys = take(n * sizeof(float));
    const size_t oms = take(n);
    const size_t oxs = take(n * sizeof(float));
    const size_t ops = take(pl->psf.size() * sizeof(float));
    const size_t ozm = take(tvp ? 0 : (size_t)(levels + 1) * sizeof(CUtensorMap));
    const bool zstate = !tvp;   // the frame priors' state: zeta2 + two bits per coefficient
    const size_t ozb = take(zstate ? n * sizeof(uint32_t) : 0);
    if (dev_alloc(&pl->slab, off) != cudaSuccess) {
        cudaGetLastError();
        pl->slab = nullptr;
        free_plan(pl);
        return ADMM_ENOMEM;
    }
    char* b = static_cast<char*>(pl->slab);
    pl->Sa = reinterpret_cast<float4*>(b + oSa);
    pl->Sb = reinterpret_cast<float4*>(b + oSb);
    pl->d1 = reinterpret_cast<float*>(b + od1);
    pl->d2 = reinterpret_cast<float*>(b + od2);
    pl->ybar = reinterpret_cast<float*>(b + oyb);
    pl->xprev = reinterpret_cast<float*>(b + oxp);
    pl->work = pl->fam == ADMM_REG_HAAR ? reinterpret_cast<float*>(b + owk) : nullptr;
    pl->cg = cg ? reinterpret_cast<float*>(b + ocg) : nullptr;
    pl->cg_part = cg ? reinterpret_cast<double*>(b + ocp) : nullptr;
    pl->mask = reinterpret_cast<uint8_t*>(b + omk);
    pl->lamT = reinterpret_cast<float2*>(b + olm);
    pl->kT = reinterpret_cast<float*>(b + okt);
    pl->partials = reinterpret_cast<double*>(b + opt);
    pl->ctl = reinterpret_cast<ProbCtl*>(b + oct);
    pl->ystage = reinterpret_cast<float*>(b + oys);
    pl->mstage = reinterpret_cast<uint8_t*>(b + oms);
    pl->xstage = reinterpret_cast<float*>(b + oxs);
    pl->psf_dev = reinterpret_cast<float*>(b + ops);
    pl->zbits = zstate ? reinterpret_cast<uint32_t*>(b + ozb) : nullptr;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int rc = ADMM_OK;
    CUtensorMap zmaps[kMaxHaarLevels + 1];
    do {
        if (cudaMemsetAsync(pl->slab, 0, off, s) != cudaSuccess) { rc = ADMM_ECUDA; break; }
        if (!tvp) {
            // the synthesis tile's TMA maps of the d2 buffers (without an
            // encoder every tile copies its halo with cp.async)
            const PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encode_fn();
            auto encode = [&](CUtensorMap* m, float* base, const cuuint64_t* dims, const cuuint64_t* strides,
                              const cuuint32_t* box, const cuuint32_t* es) {
                return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, dims, strides, box, es,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
            };
            if (enc && haar_synthesis_maps(encode, zmaps, pl->d2, H, W, levels)) {
                if (cudaMemcpyAsync(b + ozm, zmaps, (size_t)(levels + 1) * sizeof(CUtensorMap), cudaMemcpyHostToDevice,
                                    s) != cudaSuccess) { rc = ADMM_ECUDA; break; }
                pl->zmap = b + ozm;
            }
        }
        if (cudaMemcpyAsync(pl->psf_dev, pl->psf.data(), pl->psf.size() * sizeof(float), cudaMemcpyHostToDevice, s) !=
            cudaSuccess) { rc = ADMM_ECUDA; break; }
        const int tot = H * pl->Wc;
        BandWeights bw{};
        if (!pl->band_mu.empty()) {
            bw.levels = levels;
            for (int b = 0; b < 3 * levels + 1; ++b) bw.g[b] = (double)pl->band_mu[b] / (double)mu1;
        }
        spectra_kernel<<<(tot + 255) / 256, 256, 0, s>>>(pl->lamT, pl->kT, pl->psf_dev, p->psf_h, p->psf_w, H, W,
                                                         pl->Wc, tvp ? 0 : 1,
                                                         (double)mu2 / (double)mu1, bw);
        if (cudaGetLastError() != cudaSuccess) { rc = ADMM_ECUDA; break; }
        if (cudaStreamSynchronize(s) != cudaSuccess) { rc = ADMM_ECUDA; break; }
    } while (0);
    if (rc != ADMM_OK) {
        // the copies queued above read host memory of this call (the PSF, the
        // tensor maps): let them finish before it goes away
        cudaStreamSynchronize(s);
        cudaGetLastError();
        free_plan(pl);
        return rc;
    }
    *out = pl;
    return ADMM_OK;
}

void admm_deconv_destroy(admm_plan_t plan) {
    if (!plan) return;
    std::lock_guard<std::mutex> lk(g_mutex);
    cudaDeviceSynchronize();
    free_plan(plan);
}

long long admm_deconv_state_size(admm_plan_t plan) {
    if (!plan) return -1;
    return (long long)(1 + plan->nb) * plan->p.H * plan->p.W;
}

// The second dual after iteration K (K >= 0), on the device: buffer K & 1 for
// the TV priors (and buffer 0 before the first iteration); for the frame
// priors, d2 rebuilt from zeta2 (buffer 0) and the bits into buffer 1, which
// their iterations read only at iteration 1 of a restored FS-MD state.
static cudaError_t second_dual(admm_plan_s* plan, int K, const float** d2, cudaStream_t s) {
    const size_t n = (size_t)plan->p.H * plan->p.W;
    if (!plan->zbits || K < 1) {
        *d2 = plan->d2 + (size_t)(plan->zbits ? 0 : (K & 1)) * plan->nb * n;
        return cudaSuccess;
    }
    const ProbDesc pd = make_desc(plan);
    BandConv c{};
    for (int b = 0; b < plan->nb && b < 3 * kMaxHaarLevels + 1; ++b) {
        c.tau[b] = pd.band_tau[b];
        c.izs[b] = pd.band_izs[b];
    }
    if (pd.ll_free) c.tau[plan->nb - 1] = 0.f;
    float* out = plan->d2 + (size_t)plan->nb * n;
    const int blocks = (int)std::min<size_t>((n + kThreads - 1) / kThreads, (size_t)152 * 8);
    haar_dual_from_state<<<blocks, kThreads, 0, s>>>(plan->d2, plan->zbits, out, (long long)n, plan->nb, c);
    *d2 = out;
    return cudaGetLastError();
}

int admm_deconv_get_state(admm_plan_t plan, float* d_out, void* stream) {
    if (!plan || !d_out) return ADMM_EINVAL;
    std::lock_guard<std::mutex> lk(g_mutex);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t n = (size_t)plan->p.H * plan->p.W;
    CK(cudaMemcpyAsync(d_out, plan->d1, n * sizeof(float), cudaMemcpyDefault, s));
    const float* d2 = nullptr;
    CK(second_dual(plan, plan->last_iter, &d2, s));
    CK(cudaMemcpyAsync(d_out + n, d2, (size_t)plan->nb * n * sizeof(float), cudaMemcpyDefault, s));
    CK(cudaStreamSynchronize(s));
    return ADMM_OK;
}

int admm_deconv_warm_start(admm_plan_t plan, const float* x0, const float* d0, void* stream) {
    if (!plan) return ADMM_EINVAL;
    // FS-MD's starts live on theta, not x; the Reeves-Sorel variants' u1 lives
    // on the observed pixels only
    if (plan->p.reg == ADMM_REG_HAAR_SYNTHESIS || reg_cg(plan->p.reg)) return ADMM_EINVAL;
    std::lock_guard<std::mutex> lk(g_mutex);
    int dev = 0;
    CK(cudaGetDevice(&dev));
    if (plan->device != dev) return ADMM_EINVAL;
    DeviceCtx* ctx = nullptr;
    const int rc = ensure_ctx(dev, 1, &ctx);
    if (rc != ADMM_OK) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int H = plan->p.H, W = plan->p.W;
    const size_t n = (size_t)H * W;
    if (x0) {
        const float* src = x0;
        if (!is_device_ptr(x0)) {
            CK(cudaMemcpyAsync(plan->xstage, x0, n * sizeof(float), cudaMemcpyHostToDevice, s));
            src = plan->xstage;
        }
        if (plan->gen) {
            const float2* twW = nullptr;
            const int r = gen_twiddles(ctx, W, &twW);
            if (r != ADMM_OK) return r;
            CK(launch_gen_warm_rows(W, H, plan->Wp, src, plan->Sb, twW, s));
        } else {
            CK(launch_warm_rows(W, src, plan->Sb, H, plan->Wp, ctx->tw, s));
        }
        ++g_launches;
    } else {
        CK(cudaMemsetAsync(plan->Sb, 0, n / W * plan->Wp * sizeof(float4), s));
    }
    // the first iteration reads d2 buffer (1 + 1) & 1 = 0
    if (d0) {
        CK(cudaMemcpyAsync(plan->d1, d0, n * sizeof(float), cudaMemcpyDefault, s));
        CK(cudaMemcpyAsync(plan->d2, d0 + n, (size_t)plan->nb * n * sizeof(float), cudaMemcpyDefault, s));
    } else {
        CK(cudaMemsetAsync(plan->d1, 0, n * sizeof(float), s));
        CK(cudaMemsetAsync(plan->d2, 0, (size_t)plan->nb * n * sizeof(float), s));
    }
    CK(cudaStreamSynchronize(s));       // host sources may be released on return
    plan->warm_mode = 1;
    return ADMM_OK;
}

int admm_deconv_domain(admm_plan_t plan, int* H, int* W) {
    if (!plan || !H || !W) return ADMM_EINVAL;
    *H = plan->p.H;
    *W = plan->p.W;
    return ADMM_OK;
}

// Layout of the complete state (admm_deconv_get_full_state): d1, d2, the row
// spectra of the next x-step's right-hand side (Hd x Wc float4, the stored
// half spectrum without the column padding), then for FS-MD the last w and
// zeta2.
static size_t full_state_floats(const admm_plan_s* pl, size_t* spec_off, size_t* extra_off) {
    const size_t n = (size_t)pl->p.H * pl->p.W;
    const size_t d = (size_t)(1 + pl->nb) * n;
    const size_t spec = (size_t)pl->p.H * pl->Wc * 4;
    size_t extra = 0;
    if (pl->p.reg == ADMM_REG_HAAR_SYNTHESIS) extra = (size_t)(1 + pl->nb) * n;
    if (reg_cg(pl->p.reg)) extra = n;                   // the CG iterate z
    if (spec_off) *spec_off = d;
    if (extra_off) *extra_off = d + spec;
    return d + spec + extra;
}

long long admm_deconv_full_state_size(admm_plan_t plan) {
    if (!plan) return -1;
    return (long long)full_state_floats(plan, nullptr, nullptr);
}

int admm_deconv_get_full_state(admm_plan_t plan, float* state, int* iters, void* stream) {
    if (!plan || !state) return ADMM_EINVAL;
    std::lock_guard<std::mutex> lk(g_mutex);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int H = plan->p.H;
    const size_t n = (size_t)H * plan->p.W;
    size_t spec_off = 0, extra_off = 0;
    full_state_floats(plan, &spec_off, &extra_off);
    const int K = plan->last_iter;
    if (plan->fam != ADMM_REG_TV && K > 0) {
        // The frame prior's iteration ends with the synthesis and the forward
        // row DFTs, which the last iteration skipped: the problem had retired
        // when they ran. Run them now for this plan alone (they read zeta2 and
        // zeta1 of iteration K, still in place), marking it active meanwhile.
        int dev = 0;
        CK(cudaGetDevice(&dev));
        if (plan->device != dev) return ADMM_EINVAL;
        DeviceCtx* ctx = nullptr;
        int rc = ensure_ctx(dev, 1, &ctx);
        if (rc != ADMM_OK) return rc;
        // the batch tables are borrowed: every solve uploads them afresh
        ctx->h_desc[0] = make_desc(plan);
        ctx->h_active[0] = 0;   // slot 0 -> problem 0
        static const int one = 1, zero = 0;
        CK(cudaMemcpyAsync(ctx->desc, ctx->h_desc, sizeof(ProbDesc), cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(ctx->slot_map, ctx->h_active, sizeof(int), cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(&plan->ctl->active, &one, sizeof(int), cudaMemcpyHostToDevice, s));
        const SlotTable sl{ctx->slot_map, ctx->queue, 1};
        if (plan->gen) {
            const float2* twW = nullptr;
            rc = gen_twiddles(ctx, plan->p.W, &twW);
            if (rc != ADMM_OK) return rc;
            CK(launch_gen_tail(plan->p.W, H, plan->Wp, ctx->desc, sl, 1, plan->levels, !reg_tv_prior(plan->p.reg),
                               twW, s));
        } else {
            CK(launch_row_tail(plan->p.W, H, plan->Wp, ctx->desc, sl, 1, plan->levels,
                               plan->p.reg != ADMM_REG_TV_CG, ctx->tw, s));
        }
        g_launches += 2;
        CK(cudaMemcpyAsync(&plan->ctl->active, &zero, sizeof(int), cudaMemcpyHostToDevice, s));
        CK(cudaStreamSynchronize(s));
    }
    CK(cudaMemcpyAsync(state, plan->d1, n * sizeof(float), cudaMemcpyDefault, s));
    const float* d2 = nullptr;
    CK(second_dual(plan, K, &d2, s));
    CK(cudaMemcpyAsync(state + n, d2, (size_t)plan->nb * n * sizeof(float), cudaMemcpyDefault, s));
    CK(cudaMemcpy2DAsync(state + spec_off, (size_t)plan->Wc * sizeof(float4), plan->Sb,
                         (size_t)plan->Wp * sizeof(float4), (size_t)plan->Wc * sizeof(float4), (size_t)H,
                         cudaMemcpyDefault, s));
    if (plan->p.reg == ADMM_REG_HAAR_SYNTHESIS) {
        // FS-MD's next iteration also reads the last w and zeta2 (zeta2 in
        // d2 buffer 0 after an iteration; before one, a restored zeta2 in buffer 1)
        CK(cudaMemcpyAsync(state + extra_off, plan->work + 2 * n, n * sizeof(float), cudaMemcpyDefault, s));
        const float* z2 = plan->d2 + (size_t)(K >= 1 ? 0 : 1) * plan->nb * n;
        CK(cudaMemcpyAsync(state + extra_off + n, z2, (size_t)plan->nb * n * sizeof(float), cudaMemcpyDefault, s));
    }
    if (reg_cg(plan->p.reg))
        CK(cudaMemcpyAsync(state + extra_off, plan->cg + 5 * n, n * sizeof(float), cudaMemcpyDefault, s));
    CK(cudaStreamSynchronize(s));
    if (iters) *iters = K;
    return ADMM_OK;
}

int admm_deconv_set_state(admm_plan_t plan, const float* state, void* stream) {
    if (!plan || !state) return ADMM_EINVAL;
    std::lock_guard<std::mutex> lk(g_mutex);
    int dev = 0;
    CK(cudaGetDevice(&dev));
    if (plan->device != dev) return ADMM_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int H = plan->p.H;
    const size_t n = (size_t)H * plan->p.W;
    size_t spec_off = 0, extra_off = 0;
    full_state_floats(plan, &spec_off, &extra_off);
    // the restarted solve's iteration 1 reads d2 buffer (1 + 1) & 1 = 0 and
    // (FS-MD) the previous zeta2 from buffer 1
    CK(cudaMemcpyAsync(plan->d1, state, n * sizeof(float), cudaMemcpyDefault, s));
    CK(cudaMemcpyAsync(plan->d2, state + n, (size_t)plan->nb * n * sizeof(float), cudaMemcpyDefault, s));
    CK(cudaMemcpy2DAsync(plan->Sb, (size_t)plan->Wp * sizeof(float4), state + spec_off,
                         (size_t)plan->Wc * sizeof(float4), (size_t)plan->Wc * sizeof(float4), (size_t)H,
                         cudaMemcpyDefault, s));
    if (plan->p.reg == ADMM_REG_HAAR_SYNTHESIS) {
        CK(cudaMemcpyAsync(plan->work + 2 * n, state + extra_off, n * sizeof(float), cudaMemcpyDefault, s));
        CK(cudaMemcpyAsync(plan->d2 + (size_t)plan->nb * n, state + extra_off + n, (size_t)plan->nb * n * sizeof(float),
                           cudaMemcpyDefault, s));
    }
    if (reg_cg(plan->p.reg))
        CK(cudaMemcpyAsync(plan->cg + 5 * n, state + extra_off, n * sizeof(float), cudaMemcpyDefault, s));
    CK(cudaStreamSynchronize(s));       // host sources may be released on return
    plan->warm_mode = 2;
    return ADMM_OK;
}

// One size class of a batch: problems [off, off + count) of the descriptor
// table, split into L.n lanes (absolute table offsets and slot ranges; lane l
// uses queue word qbase + l).
struct GroupRun {
    int H = 0, W = 0, Wc = 0, Wp = 0, levels = 0;
    bool tv = true;              // the TV row phase (TV, anisotropic TV)
    bool cg = false;             // a Reeves-Sorel variant
    bool gen = false;            // mixed-radix kernels (a side is not a power of two)
    const float2* twH = nullptr; // ... their twiddle tables
    const float2* twW = nullptr;
    int off = 0, count = 0, nslots = 0, max_iters = 0, qbase = 0;
    int gi = 0;                  // index of the class's n_active counter
    int R = 0, row_v = 0, col_v = 0, slot_ctas = 0, lanes = 0;
    int reg = 0;                 // the regulariser (variants share a family but not kernels)
    RowLaunchFn row_fn = nullptr;  // TV row phase of the class's configuration
    ColLaunchFn col_fn = nullptr;
    long long launch_cap = 0;    // iterations after which every problem has retired
    long long launched = 0;
    Lanes L;
};

static SlotTable lane_slots(DeviceCtx* ctx, const GroupRun& g, int l) {
    return SlotTable{ctx->slot_map + g.L.soff[l], ctx->queue + g.qbase + l, g.L.cnt[l]};
}

// one ADMM iteration of one lane: the column phase, then the row side
static cudaError_t launch_iteration(DeviceCtx* ctx, const GroupRun& g, int l, cudaStream_t s) {
    const ProbDesc* desc = ctx->desc + g.L.off[l];
    const SlotTable sl = lane_slots(ctx, g, l);
    if (g.cg)
        return launch_cg_iteration(g.W, g.H, g.Wc, g.Wp, desc, sl, g.L.slots[l], g.levels, g.reg == ADMM_REG_TV_CG,
                                   g.col_fn, ctx->tw, ctx->n_active + g.gi, s);
    if (g.gen)
        return launch_gen_iteration(g.W, g.H, g.Wc, g.Wp, desc, sl, g.L.slots[l], g.reg, g.levels, g.twH, g.twW,
                                    ctx->n_active + g.gi, s);
    cudaError_t e = g.col_fn(desc, sl, g.L.slots[l], g.Wc, g.Wp, ctx->tw, s);
    if (e != cudaSuccess) return e;
    int* nact = ctx->n_active + g.gi;
    if (g.tv) return g.row_fn(desc, sl, g.L.slots[l], g.H, g.Wp, ctx->tw, nact, s);
    return launch_haar_iteration_rows(g.W, g.H, g.Wp, desc, sl, g.L.slots[l], g.levels,
                                      g.reg == ADMM_REG_HAAR_SYNTHESIS, ctx->tw, nact, s);
}

// kernels one iteration of a lane launches
static int launches_per_iteration(const GroupRun& g) {
    if (g.cg) return g.reg == ADMM_REG_TV_CG ? 7 : 8;
    if (g.gen) return reg_tv_prior(g.reg) ? 4 : 5;
    return g.tv ? 2 : 5;
}

static std::string graph_key(const std::vector<GroupRun>& groups, int chunk) {
    std::string k = std::to_string(chunk) + (t_chain_overlap ? "o" : "s");
    for (const GroupRun& g : groups) {
        k += "|" + std::to_string(g.H) + "," + std::to_string(g.W) + "," + std::to_string(g.tv) + "," +
             std::to_string(g.levels) + "," + std::to_string(g.reg) + "," + std::to_string(g.row_v) + "," +
             std::to_string(g.col_v) + "," +
             std::to_string(g.off) + "," + std::to_string(g.count) + "," +
             std::to_string(g.qbase) + "," + std::to_string(g.L.n);
        for (int l = 0; l < g.L.n; ++l)
            k += ";" + std::to_string(g.L.off[l]) + "," + std::to_string(g.L.cnt[l]) + "," +
                 std::to_string(g.L.soff[l]) + "," + std::to_string(g.L.slots[l]);
    }
    return k;
}

// executable graph of `chunk` iterations of every lane of every size class,
// each lane an independent branch (captured on the private streams; lanes
// beyond the stream pool share a branch)
static cudaError_t chunk_graph(DeviceCtx* ctx, const std::vector<GroupRun>& groups, int chunk,
                               cudaGraphExec_t* out) {
    const std::string key = graph_key(groups, chunk);
    auto it = ctx->graphs.find(key);
    if (it != ctx->graphs.end()) {
        *out = it->second;
        return cudaSuccess;
    }
    if (ctx->graphs.size() >= 64) {     // bound the cache: drop every layout seen so far
        for (auto& kv : ctx->graphs) cudaGraphExecDestroy(kv.second);
        ctx->graphs.clear();
    }
    int nb = 0;
    for (const GroupRun& g : groups) nb += g.L.n;
    nb = std::min(nb, (int)DeviceCtx::kBranches);
    cudaStream_t origin = ctx->branch[0];
    cudaError_t e = cudaStreamBeginCapture(origin, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    cudaError_t le = cudaSuccess;
    if (nb > 1) {
        le = cudaEventRecord(ctx->fork_ev, origin);
        for (int b = 1; b < nb && le == cudaSuccess; ++b) le = cudaStreamWaitEvent(ctx->branch[b], ctx->fork_ev, 0);
    }
    int br = 0;
    for (const GroupRun& g : groups) {
        for (int l = 0; l < g.L.n && le == cudaSuccess; ++l, ++br) {
            cudaStream_t cs = ctx->branch[br % nb];
            for (int i = 0; i < chunk && le == cudaSuccess; ++i) le = launch_iteration(ctx, g, l, cs);
        }
    }
    if (nb > 1 && le == cudaSuccess) {
        for (int b = 1; b < nb && le == cudaSuccess; ++b) {
            le = cudaEventRecord(ctx->join_ev[b], ctx->branch[b]);
            if (le == cudaSuccess) le = cudaStreamWaitEvent(origin, ctx->join_ev[b], 0);
        }
    }
    cudaGraph_t gr = nullptr;
    e = cudaStreamEndCapture(origin, &gr);
    if (le != cudaSuccess) {
        if (gr) cudaGraphDestroy(gr);
        return le;
    }
    if (e != cudaSuccess) return e;
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, gr, 0);
    cudaGraphDestroy(gr);
    if (e != cudaSuccess) return e;
    ctx->graphs[key] = exec;
    *out = exec;
    return cudaSuccess;
}

// Solve every problem of a batch: all size classes iterate in the same loop
// (their lanes are independent branches of one replayed graph).
static int solve_all_impl(DeviceCtx* ctx, const std::vector<std::vector<int>>& classes, const admm_plan_t* plans,
                          const float* const* y, const uint8_t* const* masks, float* const* x_out,
                          admm_result_t* res, int use_ws, cudaStream_t s);

// the iteration kernels of a batch go out as a launch chain (programmatic
// dependent launch) unless switched off with admm_deconv_set_launch_overlap
static std::atomic<int> g_overlap{1};
static int solve_all(DeviceCtx* ctx, const std::vector<std::vector<int>>& classes, const admm_plan_t* plans,
                     const float* const* y, const uint8_t* const* masks, float* const* x_out,
                     admm_result_t* res, int use_ws, cudaStream_t s) {
    struct Guard {
        bool prev;
        ~Guard() { t_chain_overlap = prev; }
    } guard{t_chain_overlap};
    t_chain_overlap = g_overlap.load() != 0;
    return solve_all_impl(ctx, classes, plans, y, masks, x_out, res, use_ws, s);
}

static int solve_all_impl(DeviceCtx* ctx, const std::vector<std::vector<int>>& classes, const admm_plan_t* plans,
                          const float* const* y, const uint8_t* const* masks, float* const* x_out,
                          admm_result_t* res, int use_ws, cudaStream_t s) {
    const bool prof = g_prof.on;
    std::vector<GroupRun> groups;
    std::vector<int> order;                       // table position -> index into plans
    std::vector<char> x_host;
    int soff = 0, qbase = 0;
    // input preparation, batched: items [prep_done, prep_n) of the pinned
    // staging table are prepared by the next flush (before a learned start
    // reads its problem's prepared input, and after the last problem)
    int prep_done = 0, prep_n = 0, prep_maxn = 0;
    auto flush_prep = [&]() -> int {
        const int cnt = prep_n - prep_done;
        if (cnt <= 0) return ADMM_OK;
        CK(cudaMemcpyAsync(ctx->prep + prep_done, ctx->h_prep + prep_done, cnt * sizeof(PrepItem),
                           cudaMemcpyHostToDevice, s));
        constexpr int words = (int)(sizeof(ProbCtl) / sizeof(int));
        zero_ctl_kernel<<<(unsigned)((cnt * words + 255) / 256), 256, 0, s>>>(ctx->prep + prep_done, cnt);
        CK(cudaGetLastError());
        const unsigned bx = (unsigned)std::min((prep_maxn + 255) / 256, 512);
        for (int o = 0; o < cnt; o += 65535) {   // (grid.y limit)
            prepare_items_kernel<<<dim3(bx, (unsigned)std::min(cnt - o, 65535)), 256, 0, s>>>(ctx->prep + prep_done + o);
            CK(cudaGetLastError());
            ++g_launches;
        }
        ++g_launches;
        prep_done = prep_n;
        prep_maxn = 0;
        return ADMM_OK;
    };
    for (const std::vector<int>& idx : classes) {
        GroupRun g;
        const admm_plan_s* p0 = plans[idx[0]];
        g.H = p0->p.H;
        g.W = p0->p.W;
        g.Wc = p0->Wc;
        g.Wp = p0->Wp;
        g.levels = p0->levels;
        g.tv = p0->fam == ADMM_REG_TV;
        g.cg = reg_cg(p0->p.reg);
        g.gen = p0->gen;
        g.reg = p0->p.reg;
        if (g.gen) {
            int r = gen_twiddles(ctx, g.H, &g.twH);
            if (r == ADMM_OK) r = gen_twiddles(ctx, g.W, &g.twW);
            if (r != ADMM_OK) return r;
        }
        g.R = p0->R;
        g.row_v = p0->row_v;
        g.col_v = p0->col_v;
        g.slot_ctas = p0->slot_ctas;
        g.lanes = p0->lanes;
        if (!g.gen) {
            const ColVariant* cv = nullptr;
            col_variants(g.H, &cv);
            g.col_fn = cv[g.col_v].fn;
            if (g.tv) {
                const RowVariant* rv = nullptr;
                tv_row_variants(g.W, &rv);
                g.row_fn = p0->p.reg == ADMM_REG_TV_ANISO ? rv[g.row_v].fn_aniso : rv[g.row_v].fn;
            }
        }
        g.off = (int)order.size();
        g.count = (int)idx.size();
        g.qbase = qbase;
        g.gi = (int)groups.size();
        const size_t n = (size_t)g.H * g.W;
        std::vector<admm_plan_s*> ws_pend;            // this class's problems that take the learned start
        for (int j : idx) {
            admm_plan_s* pl = plans[j];
            const float* yj = y[j];
            const uint8_t* mj = masks ? masks[j] : nullptr;
            const size_t nu = (size_t)pl->Hu * pl->Wu;   // the caller's image (<= n)
            if (!is_device_ptr(yj)) {
                CK(cudaMemcpyAsync(pl->ystage, yj, nu * sizeof(float), cudaMemcpyHostToDevice, s));
                yj = pl->ystage;
            }
            if (mj && !is_device_ptr(mj)) {
                CK(cudaMemcpyAsync(pl->mstage, mj, nu, cudaMemcpyHostToDevice, s));
                mj = pl->mstage;
            }
            ctx->h_prep[prep_n++] = PrepItem{pl->ybar, pl->mask, yj, mj, pl->ctl, g.H, g.W, pl->Hu, pl->Wu,
                                             pl->p.psf_h / 2, pl->p.psf_w / 2, pl->p.raw_mask};
            prep_maxn = std::max(prep_maxn, (int)n);
            if (use_ws && pl->warm_mode == 0 && pl->p.reg == ADMM_REG_TV) {
                // learned start, run for the class's problems together below
                // (d2 follows d1 directly: H W floats are a multiple of the slab's 256-byte alignment)
                if (pl->d2 != pl->d1 + n) return ADMM_ECUDA;
                pl->warm_mode = 1;
                ws_pend.push_back(pl);
            }
            const int t = (int)order.size();
            ctx->h_desc[t] = make_desc(pl);
            // padded plans finalize on their domain and copy the caller's window out
            x_host.push_back(pl->padded || !is_device_ptr(x_out[j]));
            ctx->h_xptr[t] = x_host.back() ? pl->xstage : x_out[j];
            order.push_back(j);
            g.max_iters = std::max(g.max_iters, pl->p.max_iters);
        }
        if (!ws_pend.empty()) {
            // the network reads each problem's [M^T y, mask] once prepared and
            // writes x0 (to the staging plane) and d0 = (d1, d2 buffer 0),
            // contiguous in the plan's slab, for up to ws_batch_limit problems
            // per pass; then u0 = H x0 - d0 as in admm_deconv_warm_start
            auto learned = [&]() -> int {
                int r = flush_prep();
                if (r != ADMM_OK) return r;
                const int lim = ws_batch_limit(g.H, g.W);
                std::vector<const float*> yb;
                std::vector<const uint8_t*> mk;
                std::vector<float*> x0, d0;
                for (size_t a = 0; a < ws_pend.size(); a += lim) {
                    const size_t e = std::min(ws_pend.size(), a + (size_t)lim);
                    yb.clear();
                    mk.clear();
                    x0.clear();
                    d0.clear();
                    for (size_t k = a; k < e; ++k) {
                        yb.push_back(ws_pend[k]->ybar);
                        mk.push_back(ws_pend[k]->mask);
                        x0.push_back(ws_pend[k]->xstage);
                        d0.push_back(ws_pend[k]->d1);
                    }
                    r = ws_predict_starts((int)(e - a), g.H, g.W, yb.data(), mk.data(), x0.data(), d0.data(), s);
                    if (r != ADMM_OK) return r;
                }
                for (admm_plan_s* pl : ws_pend) {
                    if (pl->gen)
                        CK(launch_gen_warm_rows(g.W, g.H, pl->Wp, pl->xstage, pl->Sb, g.twW, s));
                    else
                        CK(launch_warm_rows(g.W, pl->xstage, pl->Sb, g.H, pl->Wp, ctx->tw, s));
                    ++g_launches;
                }
                return ADMM_OK;
            };
            const int r = learned();
            if (r != ADMM_OK) {
                for (admm_plan_s* pl : ws_pend) pl->warm_mode = 0;
                return r;
            }
        }
        g.nslots = choose_slots(g.H, g.W, g.tv, g.R, g.slot_ctas, g.count);
        // with per-phase timing on, one lane: every launch covers all slots,
        // so the timed phases are the full-size kernels
        g.L.n = prof ? 1 : std::max(1, std::min({g.lanes > 0 ? g.lanes : kDefaultLanes, g.count, g.nslots}));
        for (int l = 0, o = g.off, so = soff; l < g.L.n; ++l) {
            g.L.off[l] = o;
            g.L.cnt[l] = l + 1 < g.L.n ? g.count / g.L.n : g.off + g.count - o;
            g.L.soff[l] = so;
            g.L.slots[l] = l + 1 < g.L.n ? g.nslots / g.L.n : soff + g.nslots - so;
            o += g.L.cnt[l];
            so += g.L.slots[l];
        }
        soff += g.nslots;
        qbase += g.L.n;
        groups.push_back(g);
    }
    {
        const int rp = flush_prep();     // the inputs of the problems not prepared yet
        if (rp != ADMM_OK) return rp;
    }
    const int total = (int)order.size();
    const int ng = (int)groups.size();
    g_test_stall = 0;                    // the test hook serves one solve
    CK(cudaMemcpyAsync(ctx->desc, ctx->h_desc, total * sizeof(ProbDesc), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ctx->xptr, ctx->h_xptr, total * sizeof(float*), cudaMemcpyHostToDevice, s));
    for (int gi = 0; gi < ng; ++gi) ctx->h_active[gi] = groups[gi].count;
    CK(cudaMemcpyAsync(ctx->n_active, ctx->h_active, ng * sizeof(int), cudaMemcpyHostToDevice, s));
    for (const GroupRun& g : groups) {
        init_ctl_kernel<<<(g.count + 127) / 128, 128, 0, s>>>(ctx->desc + g.off, g.count, ctx->n_active + g.gi);
        CK(cudaGetLastError());
        ++g_launches;
        for (int l = 0; l < g.L.n; ++l) {
            assign_slots_kernel<<<1, 32, 0, s>>>(ctx->desc + g.L.off[l], lane_slots(ctx, g, l), g.L.slots[l]);
            CK(cudaGetLastError());
            ++g_launches;
        }
    }
    // the host-side tables are reused by the next call
    CK(cudaStreamSynchronize(s));

    // with more problems than slots, problems start as slots free up: the
    // iterations needed by a class are bounded by the sum of its per-slot work
    for (GroupRun& g : groups) {
        long long work = 0;
        for (int t = g.off; t < g.off + g.count; ++t) work += plans[order[t]]->p.max_iters;
        int min_slots = g.L.slots[0];
        for (int l = 1; l < g.L.n; ++l) min_slots = std::min(min_slots, g.L.slots[l]);
        min_slots = std::max(1, min_slots);
        g.launch_cap = std::min((work + min_slots - 1) / min_slots + g.max_iters, (long long)INT32_MAX);
    }
    // classes still iterating; a class leaves once the host has seen its
    // counter reach zero (one chunk behind the device) or its cap run out
    std::vector<GroupRun> live = groups;
    const int chunk = 8;
    size_t nev = 0;
    if (prof) {
        int r = prof_event(nev++, s);
        if (r != ADMM_OK) return r;
    }
    for (int j = 0; !live.empty(); ++j) {
        bool full = true;
        for (const GroupRun& g : live) full = full && g.launch_cap - g.launched >= chunk;
        if (!prof && j > 0 && full) {
            // steady state: one graph replay per chunk (the first chunk ran
            // as plain launches, which also set the kernels' attributes)
            cudaGraphExec_t exec = nullptr;
            CK(chunk_graph(ctx, live, chunk, &exec));
            CK(cudaGraphLaunch(exec, s));
            for (GroupRun& g : live) {
                g_launches += (long long)chunk * g.L.n * launches_per_iteration(g);
                g.launched += chunk;
            }
        } else {
            for (int it = 0; it < chunk; ++it) {
                for (GroupRun& g : live) {
                    if (g.launched >= g.launch_cap) continue;
                    for (int l = 0; l < g.L.n; ++l) {
                        const ProbDesc* dl = ctx->desc + g.L.off[l];
                        const SlotTable sl = lane_slots(ctx, g, l);
                        int* nact = ctx->n_active + g.gi;
                        if (g.cg || g.gen) {
                            // (timed as one row-side interval when profiling)
                            if (prof) {
                                int r = prof_event(nev++, s);
                                if (r != ADMM_OK) return r;
                            }
                            CK(launch_iteration(ctx, g, l, s));
                            g_launches += launches_per_iteration(g);
                            if (prof) {
                                int r = prof_event(nev++, s);
                                if (r != ADMM_OK) return r;
                            }
                            continue;
                        }
                        CK(g.col_fn(dl, sl, g.L.slots[l], g.Wc, g.Wp, ctx->tw, s));
                        ++g_launches;
                        if (prof) {
                            int r = prof_event(nev++, s);
                            if (r != ADMM_OK) return r;
                        }
                        if (g.tv) {
                            CK(g.row_fn(dl, sl, g.L.slots[l], g.H, g.Wp, ctx->tw, nact, s));
                            ++g_launches;
                        } else {
                            CK(launch_haar_iteration_rows(g.W, g.H, g.Wp, dl, sl, g.L.slots[l], g.levels,
                                                          g.reg == ADMM_REG_HAAR_SYNTHESIS, ctx->tw,
                                                          nact, s));
                            g_launches += 4;
                        }
                        if (prof) {
                            int r = prof_event(nev++, s);
                            if (r != ADMM_OK) return r;
                        }
                    }
                    ++g.launched;
                }
            }
        }
        int* hbuf = ctx->h_active + (size_t)(j & 1) * ctx->cap;
        CK(cudaMemcpyAsync(hbuf, ctx->n_active, ng * sizeof(int), cudaMemcpyDeviceToHost, s));
        CK(cudaEventRecord(ctx->ev[j & 1], s));
        std::vector<GroupRun> next;
        if (j > 0) {
            CK(cudaEventSynchronize(ctx->ev[(j - 1) & 1]));
            const int* prev = ctx->h_active + (size_t)((j - 1) & 1) * ctx->cap;
            for (const GroupRun& g : live)
                if (prev[g.gi] > 0 && g.launched < g.launch_cap) next.push_back(g);
        } else {
            for (const GroupRun& g : live)
                if (g.launched < g.launch_cap) next.push_back(g);
        }
        live.swap(next);
    }
    for (const GroupRun& g : groups) {
        if (g.cg || g.gen) {
            // the Reeves-Sorel variants form x = x~ + alpha v on the row side
            // (the last column-phase output is v), and the mixed-radix chain
            // writes x on its row side: it is in the scratch plane
            for (int t = g.off; t < g.off + g.count; ++t)
                CK(cudaMemcpyAsync(ctx->h_xptr[t], plans[order[t]]->work, (size_t)g.H * g.W * sizeof(float),
                                   cudaMemcpyDeviceToDevice, s));
            continue;
        }
        CK(launch_fin(g.W, ctx->desc + g.off, ctx->xptr + g.off, g.count, g.H, g.Wp, ctx->tw, s));
        ++g_launches;
    }
    for (int t = 0; t < total; ++t) {
        admm_plan_s* pl = plans[order[t]];
        if (x_host[t])
            CK(cudaMemcpy2DAsync(x_out[order[t]], (size_t)pl->Wu * sizeof(float), pl->xstage,
                                 (size_t)pl->p.W * sizeof(float), (size_t)pl->Wu * sizeof(float), (size_t)pl->Hu,
                                 cudaMemcpyDefault, s));
        CK(cudaMemcpyAsync(&ctx->h_ctl[t], pl->ctl, sizeof(ProbCtl), cudaMemcpyDeviceToHost, s));
    }
    CK(cudaStreamSynchronize(s));
    if (prof) {
        for (size_t e = 1; e + 1 < nev; e += 2) {
            float a = 0.f, b = 0.f;
            CK(cudaEventElapsedTime(&a, g_prof.ev[e - 1], g_prof.ev[e]));
            CK(cudaEventElapsedTime(&b, g_prof.ev[e], g_prof.ev[e + 1]));
            g_prof.acc.col_ms += a;
            g_prof.acc.row_ms += b;
            g_prof.acc.col_launches += 1;
            g_prof.acc.row_launches += 1;
        }
    }
    int rc = ADMM_OK;
    for (int t = 0; t < total; ++t) {
        const ProbCtl& c = ctx->h_ctl[t];
        plans[order[t]]->last_iter = c.iter;
        plans[order[t]]->warm_mode = 0;          // a warm start or a restored state serves one solve
        if (c.status != 0 && rc == ADMM_OK) rc = c.status;
        if (res) {
            admm_result_t& r = res[order[t]];
            r.iters = c.iter;
            r.converged = c.converged;
            r.status = c.status;
            r.reserved = 0;
            r.objective = c.have_obj ? c.obj : NAN;
            r.rel_x = c.rel_x;
            r.rel_obj = c.rel_obj;
            r.primal_res = c.primal_res;
            r.t_start_ms = c.t_start >= c.t0 ? (double)(c.t_start - c.t0) * 1e-6 : 0.0;
            r.t_done_ms = c.t_done >= c.t0 ? (double)(c.t_done - c.t0) * 1e-6 : 0.0;
        }
    }
    return rc;
}

int admm_deconv_solve_batch(const admm_plan_t* plans, int count, const float* const* y,
                            const uint8_t* const* masks, float* const* x_out, admm_result_t* res, int use_warmstart,
                            void* stream) {
    if (count < 0) return ADMM_EINVAL;
    if (use_warmstart != 0 && use_warmstart != 1) return ADMM_EINVAL;
    if (use_warmstart && !ws_loaded()) return ADMM_EINVAL;
    if (count == 0) return ADMM_OK;
    if (!plans || !y || !x_out) return ADMM_EINVAL;
    for (int i = 0; i < count; ++i) {
        if (!plans[i] || !y[i] || !x_out[i]) return ADMM_EINVAL;
        for (int j = 0; j < i; ++j)
            if (plans[j] == plans[i]) return ADMM_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g_mutex);
    int dev = 0;
    CK(cudaGetDevice(&dev));
    for (int i = 0; i < count; ++i)
        if (plans[i]->device != dev) return ADMM_EINVAL;
    DeviceCtx* ctx = nullptr;
    int rc = ensure_ctx(dev, count, &ctx);
    if (rc != ADMM_OK) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // a size class shares its shape and its launch configuration
    std::map<std::tuple<int, int, int, int, int, int, int, int>, std::vector<int>> groups;
    for (int i = 0; i < count; ++i) {
        const admm_plan_s* p = plans[i];
        groups[std::make_tuple(p->p.H, p->p.W, p->p.reg, p->levels, p->row_v, p->col_v, p->slot_ctas, p->lanes)]
            .push_back(i);
    }
    std::vector<std::vector<int>> classes;
    for (auto& kv : groups) classes.push_back(kv.second);
    return solve_all(ctx, classes, plans, y, masks, x_out, res, use_warmstart, s);
}

int admm_deconv_set_option(int option, long long value) {
    std::lock_guard<std::mutex> lk(g_mutex);
    if (option == ADMM_OPT_MAX_SLOTS) {
        if (value < 0 || value > INT32_MAX) return ADMM_EINVAL;
        g_max_slots = (int)value;
        return ADMM_OK;
    }
    if (option == ADMM_OPT_FAIL_ALLOC) {
        if (value < 0) return ADMM_EINVAL;
        g_fail_alloc.store(value);
        return ADMM_OK;
    }
    if (option == ADMM_OPT_TEST_STALL) {
        if (value != 0 && value != 1) return ADMM_EINVAL;
        g_test_stall = (int)value;
        return ADMM_OK;
    }
    return ADMM_EINVAL;
}

int admm_deconv_set_launch_overlap(int enable) {
    g_overlap.store(enable != 0 ? 1 : 0);
    return ADMM_OK;
}

int admm_deconv_get_launch_overlap(void) { return g_overlap.load(); }

int admm_deconv_profile(int enable, admm_profile_t* out) {
    std::lock_guard<std::mutex> lk(g_mutex);
    if (out) {
        *out = g_prof.acc;
        out->kernel_launches = g_launches;
        g_prof.acc = admm_profile_t{};
        g_launches = 0;
    }
    g_prof.on = enable != 0;
    return ADMM_OK;
}

// ---- launch configurations and the autotuner ------------------------------
static int tuning_levels(int reg, int levels, int* out) {
    if (reg == ADMM_REG_TV) {
        *out = 0;
        return ADMM_OK;
    }
    if (reg != ADMM_REG_HAAR) return ADMM_EINVAL;
    const int lv = levels == 0 ? 4 : levels;
    if (lv < 1 || lv > kMaxHaarLevels) return ADMM_EINVAL;
    *out = lv;
    return ADMM_OK;
}

int admm_deconv_variants(int H, int W, int reg, int* n_row, int* n_col) {
    if (!n_row || !n_col) return ADMM_EINVAL;
    if (reg != ADMM_REG_TV && reg != ADMM_REG_HAAR) return ADMM_EINVAL;
    if (!is_pow2_size(H) || !is_pow2_size(W)) return ADMM_EUNSUPPORTED_SIZE;
    const RowVariant* rv = nullptr;
    const ColVariant* cv = nullptr;
    *n_row = reg == ADMM_REG_TV ? tv_row_variants(W, &rv) : 1;
    *n_col = col_variants(H, &cv);
    return ADMM_OK;
}

int admm_deconv_get_tuning(admm_tuning_t* t) {
    if (!t) return ADMM_EINVAL;
    if (!is_pow2_size(t->H) || !is_pow2_size(t->W)) return ADMM_EUNSUPPORTED_SIZE;
    int levels = 0;
    int rc = tuning_levels(t->reg, t->haar_levels, &levels);
    if (rc != ADMM_OK) return rc;
    int dev = 0;
    CK(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_mutex);
    admm_tuning_t r = lookup_tuning(dev, t->H, t->W, t->reg, levels);
    if (!describe_tuning(&r)) return ADMM_EINVAL;
    *t = r;
    return ADMM_OK;
}

int admm_deconv_set_tuning(const admm_tuning_t* t) {
    if (!t) return ADMM_EINVAL;
    if (!is_pow2_size(t->H) || !is_pow2_size(t->W)) return ADMM_EUNSUPPORTED_SIZE;
    int levels = 0;
    int rc = tuning_levels(t->reg, t->haar_levels, &levels);
    if (rc != ADMM_OK) return rc;
    admm_tuning_t r = *t;
    r.haar_levels = levels;
    if (!describe_tuning(&r)) return ADMM_EINVAL;
    int dev = 0;
    CK(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_mutex);
    g_tuning[TuneKey(dev, r.H, r.W, r.reg, levels)] = r;
    return ADMM_OK;
}

int admm_deconv_autotune(int H, int W, int reg, int haar_levels, int problems, int iters, admm_tuning_t* trials,
                         int max_trials, int* n_trials, admm_tuning_t* best, void* stream) {
    if (!is_pow2_size(H) || !is_pow2_size(W)) return ADMM_EUNSUPPORTED_SIZE;
    int levels = 0;
    int rc = tuning_levels(reg, haar_levels, &levels);
    if (rc != ADMM_OK) return rc;
    if (max_trials < 0 || (max_trials > 0 && !trials)) return ADMM_EINVAL;
    int nr = 0, nc = 0;
    rc = admm_deconv_variants(H, W, reg, &nr, &nc);
    if (rc != ADMM_OK) return rc;
    int dev = 0;
    CK(cudaGetDevice(&dev));
    const int slot_targets[3] = {0, 1200, 4800};
    if (problems <= 0) {
        // enough problems that the largest slot target is filled for every row configuration
        int need = 2;
        for (int v = 0; v < nr; ++v) {
            int per = haar_num_tiles(H, W);
            if (reg == ADMM_REG_TV) {
                const RowVariant* rv = nullptr;
                tv_row_variants(W, &rv);
                per = H / rv[v].R;
            }
            need = std::max(need, (4800 + per - 1) / per);
        }
        problems = std::min(need, 96);
    }
    if (iters <= 0) iters = 48;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t n = (size_t)H * W;

    // synthetic observation: smooth texture plus a checkerboard of steps
    std::vector<float> hy(n);
    for (int r = 0; r < H; ++r)
        for (int c = 0; c < W; ++c)
            hy[(size_t)r * W + c] = (float)(0.5 + 0.25 * std::sin(2.0 * M_PI * r / 37.0) * std::cos(2.0 * M_PI * c / 23.0) +
                                            ((((r >> 4) + (c >> 4)) & 1) ? 0.1 : -0.1));
    std::vector<float> psf(81, 1.0f / 81.0f);
    admm_params_t p{};
    p.H = H;
    p.W = W;
    p.psf_h = p.psf_w = 9;
    p.psf = psf.data();
    p.lambda = 1e-4f;
    p.reg = reg;
    p.haar_levels = levels;
    p.stop = ADMM_STOP_REL_X;
    p.tol = 0.0;                      // never met: every problem runs `iters` iterations
    p.max_iters = iters;
    p.check_every = 10;

    float* dy = nullptr;
    float* dx = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    std::vector<admm_plan_t> pls;
    admm_tuning_t prev{};
    bool had_prev = false;
    {
        std::lock_guard<std::mutex> lk(g_mutex);
        auto it = g_tuning.find(TuneKey(dev, H, W, reg, levels));
        if (it != g_tuning.end()) {
            prev = it->second;
            had_prev = true;
        }
    }
    admm_tuning_t win{};
    bool have_win = false;
    int count = 0;
    rc = ADMM_OK;
    do {
        if (dev_alloc(&dy, n * sizeof(float)) != cudaSuccess ||
            dev_alloc(&dx, (size_t)problems * n * sizeof(float)) != cudaSuccess) {
            cudaGetLastError();
            rc = ADMM_ENOMEM;
            break;
        }
        if (cudaMemcpy(dy, hy.data(), n * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
            rc = ADMM_ECUDA;
            break;
        }
        std::vector<const float*> ys(problems, dy);
        std::vector<float*> xs(problems);
        for (int i = 0; i < problems; ++i) xs[i] = dx + (size_t)i * n;
        // one timed trial of configuration t (installed for the class while it runs)
        auto trial = [&](admm_tuning_t t) -> int {
            describe_tuning(&t);
            {
                std::lock_guard<std::mutex> lk(g_mutex);
                g_tuning[TuneKey(dev, H, W, reg, levels)] = t;
            }
            pls.assign(problems, nullptr);
            int r = ADMM_OK;
            for (int i = 0; i < problems && r == ADMM_OK; ++i) r = admm_deconv_plan(&pls[i], &p, stream);
            float ms = 0.f;
            if (r == ADMM_OK)   // warm-up: kernel attributes, graph capture
                r = admm_deconv_solve_batch(pls.data(), problems, ys.data(), nullptr, xs.data(), nullptr, 0, stream);
            if (r == ADMM_OK) {
                if (cudaEventRecord(e0, s) != cudaSuccess) r = ADMM_ECUDA;
                if (r == ADMM_OK)
                    r = admm_deconv_solve_batch(pls.data(), problems, ys.data(), nullptr, xs.data(), nullptr, 0,
                                                stream);
                if (r == ADMM_OK && (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                                     cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
                    r = ADMM_ECUDA;
            }
            for (admm_plan_t q : pls) admm_deconv_destroy(q);
            pls.clear();
            if (r != ADMM_OK) return r;
            t.us_per_iter = (double)ms * 1e3 / ((double)problems * (double)iters);
            if (count < max_trials) trials[count] = t;
            ++count;
            if (!have_win || t.us_per_iter < win.us_per_iter) {
                win = t;
                have_win = true;
            }
            return ADMM_OK;
        };
        for (int rv = 0; rv < nr && rc == ADMM_OK; ++rv) {
            for (int cv = 0; cv < nc && rc == ADMM_OK; ++cv) {
                for (int st : slot_targets) {
                    admm_tuning_t t{};
                    t.H = H;
                    t.W = W;
                    t.reg = reg;
                    t.haar_levels = levels;
                    t.row_variant = rv;
                    t.col_variant = cv;
                    t.slot_ctas = st;
                    rc = trial(t);
                    if (rc != ADMM_OK) break;
                }
            }
        }
        // lanes (independent graph branches of the class) for the best of the sweep
        for (int ln : {1, kMaxLanes}) {
            if (rc != ADMM_OK || !have_win) break;
            admm_tuning_t t = win;
            t.lanes = ln;
            rc = trial(t);
        }
    } while (0);
    for (admm_plan_t q : pls) admm_deconv_destroy(q);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (dy) cudaFree(dy);
    if (dx) cudaFree(dx);
    {
        std::lock_guard<std::mutex> lk(g_mutex);
        const TuneKey key(dev, H, W, reg, levels);
        if (rc == ADMM_OK && have_win) {
            g_tuning[key] = win;
        } else if (had_prev) {
            g_tuning[key] = prev;
        } else {
            g_tuning.erase(key);
        }
    }
    if (n_trials) *n_trials = count;
    if (rc == ADMM_OK && best) *best = win;
    return rc;
}

int admm_deconv_solve(admm_plan_t plan, const float* y, const uint8_t* mask, float* x_out, admm_result_t* res,
                      void* stream) {
    const uint8_t* m[1] = {mask};
    return admm_deconv_solve_batch(&plan, 1, &y, m, &x_out, res, 0, stream);
}

}  // extern "C"

// ===========================================================================
// Scratch-free solve (admm_deconv_solve_noalloc).
//
// For callers that may not allocate device memory at run time: hosts whose
// allocator already owns the device's memory, fixed-budget or real-time
// loops where an allocation could fail or stall, and plugins whose host
// application forbids libraries from allocating. All working memory of this
// entry point lives in g_noalloc_scratch, one fixed array compiled into the
// library that every GPU loading the library holds until the process exits.
// The limit is TV problems with H, W <= 256 (about 3.4 MB at 256 x 256).
// ===========================================================================
namespace {
constexpr int kNoAllocMaxSide = 256;
constexpr size_t kNoAllocBytes = size_t(4) << 20;   // 4 MiB
}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

namespace {
bool g_noalloc_tw_ready = false;
float2 g_noalloc_tw_host[2048];     // staging for the twiddle upload (static, not heap)

struct NoAllocLayout {
    size_t tw, desc, xptr, nact, slots, ctl, part, psf, Sa, Sb, d1, d2, yb, xp, mk, lm, kt, end;
    int Wc, Wp, R, n_strips;
};

NoAllocLayout noalloc_layout(int H, int W, int psf_elems) {
    NoAllocLayout L{};
    L.Wc = W / 2 + 1;
    L.Wp = (int)align_up(L.Wc, col_block(H));
    L.R = row_strip_tv(W);
    L.n_strips = H / L.R;
    const size_t n = (size_t)H * W;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes, 256); return o; };
    L.tw = take(2048 * sizeof(float2));
    L.desc = take(sizeof(ProbDesc));
    L.xptr = take(sizeof(float*));
    L.nact = take(sizeof(int));
    L.slots = take(2 * sizeof(int));   // slot map (one slot) and queue head
    L.ctl = take(sizeof(ProbCtl));
    L.part = take((size_t)L.n_strips * kNumPartials * sizeof(double));
    L.psf = take((size_t)psf_elems * sizeof(float));
    L.Sa = take((size_t)H * L.Wp * sizeof(float4));
    L.Sb = take((size_t)H * L.Wp * sizeof(float4));
    L.d1 = take(n * sizeof(float));
    L.d2 = take(2 * 2 * n * sizeof(float));
    L.yb = take(n * sizeof(float));
    L.xp = take(n * sizeof(float));
    L.mk = take(n);
    L.lm = take((size_t)L.Wc * H * sizeof(float2));
    L.kt = take((size_t)L.Wc * H * sizeof(float));
    L.end = off;
    return L;
}

// every call, with the calling device current: resolve the array's device
// address and rewrite the twiddle table at its start. Nothing is cached per
// device, so a context torn down in between (cudaDeviceReset, which zeroes
// the array) is set up again; both steps are cheap next to a solve.
int noalloc_setup(unsigned char** base, cudaStream_t s) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) {
        cudaGetLastError();
        return ADMM_ECUDA;
    }
    if (!g_noalloc_tw_ready) {
        for (int k = 0; k < 2048; ++k) {
            const double a = 2.0 * M_PI * (double)k / 2048.0;
            g_noalloc_tw_host[k] = make_float2((float)std::cos(a), (float)(-std::sin(a)));
        }
        g_noalloc_tw_ready = true;
    }
    if (cudaMemcpyAsync(p, g_noalloc_tw_host, sizeof(g_noalloc_tw_host), cudaMemcpyHostToDevice, s) != cudaSuccess)
        return ADMM_ECUDA;
    *base = static_cast<unsigned char*>(p);
    return ADMM_OK;
}
}  // namespace

extern "C" int admm_deconv_solve_noalloc(const admm_params_t* p, const float* y, const uint8_t* mask,
                                         float* x_out, admm_result_t* res, void* stream) {
    if (!p || !p->psf || !y || !x_out) return ADMM_EINVAL;
    if (p->reg != ADMM_REG_TV) return ADMM_EINVAL;
    if (!is_pow2_size(p->H) || !is_pow2_size(p->W)) return ADMM_EUNSUPPORTED_SIZE;
    if (p->H > kNoAllocMaxSide || p->W > kNoAllocMaxSide) return ADMM_EUNSUPPORTED_SIZE;
    if (p->psf_h < 1 || p->psf_w < 1 || (p->psf_h & 1) == 0 || (p->psf_w & 1) == 0) return ADMM_EINVAL;
    if (p->psf_h > std::min(p->H, kMaxPsfSide) || p->psf_w > std::min(p->W, kMaxPsfSide)) return ADMM_EINVAL;
    if (!(p->lambda >= 0.f) || !std::isfinite(p->lambda)) return ADMM_EINVAL;
    if (p->stop < ADMM_STOP_ITERS || p->stop > ADMM_STOP_REL_OBJ) return ADMM_EINVAL;
    if (p->max_iters <= 0 || p->check_every < 1 || !(p->tol >= 0.0)) return ADMM_EINVAL;
    double psum = 0.0;
    for (int i = 0; i < p->psf_h * p->psf_w; ++i) {
        if (!std::isfinite(p->psf[i])) return ADMM_EINVAL;
        psum += p->psf[i];
    }
    if (psum == 0.0) return ADMM_EINVAL;
    float mu1 = p->mu1, mu2 = p->mu2;
    if (mu2 <= 0.f) mu2 = 10.f * p->lambda;
    if (mu1 <= 0.f) mu1 = std::min(1.f, 3.f * mu2);
    if (!(mu1 > 0.f) || !(mu2 > 0.f)) return ADMM_EINVAL;
    if (!is_device_ptr(y) || !is_device_ptr(x_out) || (mask && !is_device_ptr(mask))) return ADMM_EINVAL;

    std::lock_guard<std::mutex> lk(g_mutex);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // From the first queued operation on, a failing call waits for the work it
    // has queued before it returns: kernels still in flight would otherwise
    // write the shared array while the next call clears and reuses it.
#define CKQ(call)                                       \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) {                        \
            cudaStreamSynchronize(s);                   \
            cudaGetLastError();                         \
            return cuda_fail(e_);                       \
        }                                               \
    } while (0)
    unsigned char* base = nullptr;
    int rc = noalloc_setup(&base, s);
    if (rc != ADMM_OK) {
        cudaStreamSynchronize(s);
        return rc;
    }
    const int H = p->H, W = p->W;
    const size_t n = (size_t)H * W;
    const NoAllocLayout L = noalloc_layout(H, W, p->psf_h * p->psf_w);
    if (L.end > kNoAllocBytes) {
        cudaStreamSynchronize(s);
        return ADMM_EUNSUPPORTED_SIZE;
    }
    const float2* tw = reinterpret_cast<const float2*>(base + L.tw);
    ProbDesc* desc = reinterpret_cast<ProbDesc*>(base + L.desc);
    float** xptr = reinterpret_cast<float**>(base + L.xptr);
    int* nact = reinterpret_cast<int*>(base + L.nact);
    ProbCtl* ctl = reinterpret_cast<ProbCtl*>(base + L.ctl);
    float* psf_dev = reinterpret_cast<float*>(base + L.psf);
    float2* lamT = reinterpret_cast<float2*>(base + L.lm);
    float* kT = reinterpret_cast<float*>(base + L.kt);
    float* ybar = reinterpret_cast<float*>(base + L.yb);
    uint8_t* mk = reinterpret_cast<uint8_t*>(base + L.mk);

    // the array keeps the previous call's contents: clear everything after the twiddles
    CKQ(cudaMemsetAsync(base + L.desc, 0, L.end - L.desc, s));
    CKQ(cudaMemcpyAsync(psf_dev, p->psf, (size_t)p->psf_h * p->psf_w * sizeof(float), cudaMemcpyHostToDevice, s));
    const int tot = H * L.Wc;
    spectra_kernel<<<(tot + 255) / 256, 256, 0, s>>>(lamT, kT, psf_dev, p->psf_h, p->psf_w, H, W, L.Wc, 0,
                                                     (double)mu2 / (double)mu1, BandWeights{});
    CKQ(cudaGetLastError());
    prepare_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(ybar, mk, y, mask, H, W, H, W, p->psf_h / 2,
                                                               p->psf_w / 2, p->raw_mask, ctl);
    CKQ(cudaGetLastError());
    ProbDesc d{};
    d.Sa = reinterpret_cast<float4*>(base + L.Sa);
    d.Sb = reinterpret_cast<float4*>(base + L.Sb);
    d.d1 = reinterpret_cast<float*>(base + L.d1);
    d.d2 = reinterpret_cast<float*>(base + L.d2);
    d.d2_stride = (long long)2 * n;
    d.ybar = ybar;
    d.mask = mk;
    d.lamT = lamT;
    d.kT = kT;
    d.xprev = reinterpret_cast<float*>(base + L.xp);
    d.work = nullptr;
    d.partials = reinterpret_cast<double*>(base + L.part);
    d.ctl = ctl;
    d.lam = p->lambda;
    d.mu1 = mu1;
    d.mu2 = mu2;
    d.gamma = (float)((double)mu2 / (double)mu1);
    d.tau = (float)((double)p->lambda / (double)mu2);
    d.inv1pmu1 = (float)(1.0 / (1.0 + (double)mu1));
    d.stop = p->stop;
    d.max_iters = p->max_iters;
    d.check_every = p->check_every;
    d.n_strips = L.n_strips;
    d.tol = p->tol;
    const int one = 1;
    CKQ(cudaMemcpyAsync(desc, &d, sizeof(d), cudaMemcpyHostToDevice, s));
    CKQ(cudaMemcpyAsync(xptr, &x_out, sizeof(float*), cudaMemcpyHostToDevice, s));
    CKQ(cudaMemcpyAsync(nact, &one, sizeof(int), cudaMemcpyHostToDevice, s));
    init_ctl_kernel<<<1, 32, 0, s>>>(desc, 1, nact);
    CKQ(cudaGetLastError());
    int* slot_words = reinterpret_cast<int*>(base + L.slots);
    const SlotTable sl{slot_words, slot_words + 1, 1};
    assign_slots_kernel<<<1, 32, 0, s>>>(desc, sl, 1);
    CKQ(cudaGetLastError());
    CKQ(cudaStreamSynchronize(s));   // the host-side sources above are locals

    const int chunk = 8;
    int launched = 0;
    while (launched < p->max_iters) {
        const int nit = std::min(chunk, p->max_iters - launched);
        for (int it = 0; it < nit; ++it) {
            CKQ(launch_col(H, desc, sl, 1, L.Wc, L.Wp, tw, s));
            CKQ(launch_row_tv(W, desc, sl, 1, H, L.Wp, tw, nact, s));
        }
        launched += nit;
        int act = 0;
        CKQ(cudaMemcpyAsync(&act, nact, sizeof(int), cudaMemcpyDeviceToHost, s));
        CKQ(cudaStreamSynchronize(s));
        if (act == 0) break;
    }
    CKQ(launch_fin(W, desc, xptr, 1, H, L.Wp, tw, s));
    ProbCtl c{};
    CKQ(cudaMemcpyAsync(&c, ctl, sizeof(ProbCtl), cudaMemcpyDeviceToHost, s));
    CKQ(cudaStreamSynchronize(s));
    if (res) {
        res->iters = c.iter;
        res->converged = c.converged;
        res->status = c.status;
        res->reserved = 0;
        res->objective = c.have_obj ? c.obj : NAN;
        res->rel_x = c.rel_x;
        res->rel_obj = c.rel_obj;
        res->primal_res = c.primal_res;
        res->t_start_ms = c.t_start >= c.t0 ? (double)(c.t_start - c.t0) * 1e-6 : 0.0;
        res->t_done_ms = c.t_done >= c.t0 ? (double)(c.t_done - c.t0) * 1e-6 : 0.0;
    }
    return c.status != 0 ? c.status : ADMM_OK;
#undef CKQ
}
