// The handle behind the C ABI and the helpers its entry points share
// (mmod_api.cu: create / model / forward; mmod_adjoint.cu: adjoint, gradient).
#pragma once
#include <string>
#include <vector>

#include "mmod_cpml.h"
#include "mmod_internal.h"
#include "tma_plan.h"

namespace mmod {

// Device-side injection table (see InjTable) plus the per-source positions
// the scale kernel reads.
struct DevInj {
    int *tile_start = nullptr, *pt_i = nullptr, *pt_j = nullptr, *pt_k = nullptr, *pt_first = nullptr;
    int *src_row = nullptr, *src_i = nullptr, *src_j = nullptr, *src_k = nullptr;
    long long *pt_off = nullptr;
    float *src_scale = nullptr;
    int npts = 0, nsrc = 0, tiles_x = 0, tiles_y = 0;
    InjTable view() const {
        InjTable t;
        t.tile_start = tile_start; t.pt_i = pt_i; t.pt_j = pt_j; t.pt_k = pt_k; t.pt_off = pt_off;
        t.pt_first = pt_first; t.src_row = src_row; t.src_scale = src_scale;
        t.tiles_x = tiles_x; t.tiles_y = tiles_y; t.npts = npts;
        return t;
    }
};

// Who injects and who is recorded: the forward run injects the sources
// (scale c / (hx hy hz)) and gathers at the receivers; the adjoint run
// injects at the receivers (scale c) and gathers at the sources.
struct Geometry {
    DevInj inj;
    long long *gather_off = nullptr;
    int ngather = 0;
    double cell = 1.0;   // divisor of the injection scale
    // gathers bucketed per (64 x 16 tile, plane) for the persistent kernel
    int *g_start = nullptr, *g_idx = nullptr;
    long long *g_off = nullptr;
};

// A cached CUDA graph of one time loop.
struct GraphSlot {
    cudaGraphExec_t exec = nullptr;
    const void *key[4] = {nullptr, nullptr, nullptr, nullptr};
    int kernel = -1;
    long long opts = -1;
    long long launches = 0;
};

}  // namespace mmod

struct mmod_handle {
    mmod_config cfg{};
    std::vector<int> src, rec;     // owned copies of the position lists
    int device = 0;
    int nxp = 0;
    long long plane = 0, vol = 0;  // padded plane / volume, in floats
    long long npts = 0;            // nx * ny * nz
    mmod::Weights w{};
    double coef[mmod::kRadius] = {};    // c_1..c_4 of the Laplacian (unit spacing)
    double symbol_max = 0.0;            // max over k of sum 2 c_m (1 - cos m k): stability bound

    float *u[2] = {nullptr, nullptr};   // wavefields (padded)
    float *c = nullptr;                 // dt^2 v^2 (padded)
    float *eta = nullptr;               // dt * eta_x | dt * eta_y | dt * eta_z
    mmod::Geometry fwd, adj;
    unsigned int *vmax_bits = nullptr;
    unsigned long long *bad = nullptr;
    float *vel_copy = nullptr;          // dense velocity of the current model (gradient scaling)

    float *st_vol = nullptr;            // dense [nz][ny][nx] staging (lazy)
    float *st_wav = nullptr;            // [nsrc][nt] staging (lazy)
    float *st_tr = nullptr;             // [nt][nrec] staging (lazy)
    float *st_adjw = nullptr;           // adjoint residual [nt][nrec], the copy the graph reads (lazy)
    float *st_adjg = nullptr;           // adjoint gathers [nt][nsrc] (lazy)
    float *st_adjo = nullptr;           // adjoint output staging [nsrc][nt] (lazy)
    int *err_host = nullptr;            // mapped pinned word: a kernel gave up waiting
    int *err_dev = nullptr;

    cudaStream_t cap = nullptr;         // private stream used only for graph capture
    cudaEvent_t ev_t0 = nullptr, ev_t1 = nullptr;   // bracket the step loop
    // Host traces download in kTraceChunks pieces while the loop runs: the
    // forward loop graph records ev_rows[i] once trace rows [0, rows_at[i])
    // are final; st_copy waits for each and copies the rows.
    static constexpr int kTraceChunks = 8;
    cudaEvent_t ev_rows[kTraceChunks] = {};
    long long rows_at[kTraceChunks] = {};
    cudaStream_t st_copy = nullptr;
    cudaEvent_t ev_copied = nullptr;
    mmod::GraphSlot g_fwd, g_adj;

    mmod::TmaPlan plans[mmod::kMaxTmaVariants]{};
    int variant = -1;                   // -1: automatic choice
    int pdl = 1;                        // MMOD_OPT_PDL (set at create)
    int persistent = 0;                 // MMOD_OPT_PERSISTENT (set at create)
    int persistent_ctas = 0;            // MMOD_OPT_PERSISTENT_CTAS (0: as many as fit)
    int test_stall = 0;                 // MMOD_OPT_TEST_STALL (one run)
    int zlen_override = 0;              // MMOD_OPT_ZLEN (0: the plan's z ranges)
    int cpml_planes = 0;                // MMOD_OPT_CPML_PLANES (0: the default)
    int claim_planes = 0;               // MMOD_OPT_CLAIM (0: the static plan)
    int *claim_ctr = nullptr;           // {next unit, CTAs done} of work-claiming step launches
    float *cpml_mem = nullptr;          // CPML: psi_x, psi_y, psi_z, zeta_x, zeta_y, zeta_z volumes
    float *cpml_bg = nullptr;           // CPML: b_x | b_y | b_z | g_x | g_y | g_z per cell
    float *cpml_xc = nullptr;           // CPML: compact x layers of the tiled pass (psi_x | zeta_x | c_x)
    long long cpml_xc_floats = 0;
    mmod::CpmlTiles cpml_tiles{};       // CPML: tensor maps of the tiled layer passes
    int cpml_tiles_on = 1;              // MMOD_OPT_CPML_TILES
    mutable mmod::TmaPlan plan_tmp;     // active_plan() with the override applied
    mutable mmod::TmaPlan plan_tmp_g;   // the same for the steps that write g^n
    int *counters = nullptr;            // per work unit of the persistent kernel
    unsigned long long *queue = nullptr;   // the persistent kernel's next (step, unit) item
    long long ncounters = 0;
    int ckpt_scheme = MMOD_SCHEME_SEGMENTS;   // MMOD_OPT_CKPT_SCHEME
    bool tma_ok = false;
    CUtensorMap cur_map[2], prev_map[2], c_map;

    // gradient work space (lazy, sized for the last checkpoint layout)
    struct GradWork {
        int nslot = 0, nwork = 0, dtype = -1;
        std::vector<float *> seg;           // nwork padded FP32 work volumes
        std::vector<CUtensorMap> seg_cur, seg_prev;
        float *psi[2] = {nullptr, nullptr};
        CUtensorMap psi_cur[2], psi_prev[2];
        float *gradc = nullptr;             // padded FP32 sum of psi^{n+1} g^n
        void *ckpt = nullptr;               // nslot * 2 volumes (FP32 or 16-bit)
        float *ckpt_scale = nullptr;        // 16-bit storage: per-plane (BF16, FP16) or per-32-value
                                            // (BFP16) scales of the nslot * 2 volumes
        size_t ckpt_bytes = 0;
    } gw;

    bool model_set = false;
    double vmax = 0.0;
    bool state_pending = false;
    bool ran = false;
    int kernel = MMOD_KERNEL_AUTO;
    long long last_launches = 0;
    cudaError_t latched = cudaSuccess;
    std::string err;
};

namespace mmod {

// Binomial checkpointing (mmod_revolve.cu): one action of a reversal
// schedule, kind = MMOD_REV_*; returns the number of advanced steps.
struct RevAction {
    int kind, a, b;
};
long long revolve_schedule(int nsteps, int snaps, std::vector<RevAction> *out);

// Shared by the entry points (mmod_api.cu).
mmod_status fail(mmod_handle *h, mmod_status st, const std::string &msg);
mmod_status fail_cuda(mmod_handle *h, cudaError_t e, const char *what);
mmod_status check_latched(mmod_handle *h);
bool is_device_ptr(const void *p);
bool use_tma(const mmod_handle *h);
int persistent_grid_of(const mmod_handle *h);
mmod_status enqueue_tune_steps(mmod_handle *h, int steps, cudaStream_t s);   // mmod_batch.cu
// Stencil weights (mmod_coeffs.cu).
bool optimized_weights(double kmax, double c[kRadius]);
double symbol_max(const double c[kRadius]);
void set_weights(mmod_handle *h, const double c[kRadius]);
void drop_graphs(mmod_handle *h);   // mmod_api.cu: captured loops must be re-captured
inline bool is_cpml(const mmod_handle *h) { return h->cfg.boundary == MMOD_BOUNDARY_CPML; }
CpmlArgs cpml_args(const mmod_handle *h);
const TmaPlan &active_plan(const mmod_handle *h);
StepArgs base_args(mmod_handle *h, const Geometry &geo, const float *wavelet);
// Enqueues one step (plain path: step, injection, optional gather of
// u^{n+1} into plain_gather_dst; TMA path: one kernel).
cudaError_t enqueue_step(mmod_handle *h, const StepArgs &a, const CUtensorMap *cur, const CUtensorMap *prev,
                         bool tma, float *plain_gather_dst, cudaStream_t s, long long *count);
// The nt-step loop of a run from u[0], u[1] with geometry geo, captured into
// the graph slot g on first use and replayed.
mmod_status run_loop_graph(mmod_handle *h, GraphSlot &g, const Geometry &geo, const float *wav, float *tr,
                           cudaStream_t s, long long *launches);

void free_grad_work(mmod_handle *h);   // mmod_adjoint.cu

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int d) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != d) cudaSetDevice(d);
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

}  // namespace mmod

#define MMOD_CK(h, call)                                              \
    do {                                                              \
        cudaError_t _e = (call);                                      \
        if (_e != cudaSuccess) return mmod::fail_cuda((h), _e, #call); \
    } while (0)
