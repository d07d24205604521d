// C ABI of the EMPSO library (include/empso.h): argument validation, the
// context (per-grid tables, workspace, swarm state) and the batch builder that
// turns (model, shot) pairs into one persistent modelling launch.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <random>
#include <map>
#include <mutex>
#include <new>
#include <sstream>
#include <string>
#include <tuple>
#include <iterator>
#include <vector>

#include "internal.cuh"

using namespace empso;

// run lengths (rows per thread) of the on-chip kernel that the planner and
// the autotuner consider, in the planner's order of preference on a tie
// (the 461 x 151 grid on 9-CTA clusters: 13 rows 568.1 G updates/s, 11 and
// 9 rows 551.1)
constexpr int RESIDENT_RUNS[] = {13, 11, 9, 8, 6};

// Occupancy answers depend only on the device and the launch shape, and the
// planner asks for every cluster size and run length of every batch (each
// surrogate generation plans a batch): memoised process-wide.
int memo_resident_clusters(int R, int C, int threads, size_t smem, int rows, bool hist = false)
{
    static std::mutex mu;
    static std::map<std::tuple<int, int, int, int, size_t, int, bool>, int> memo;
    int dev = 0;
    cudaGetDevice(&dev);
    const auto key = std::make_tuple(dev, R, C, threads, smem, rows, hist);
    std::lock_guard<std::mutex> lock(mu);
    const auto it = memo.find(key);
    if (it != memo.end()) return it->second;
    const int n = resident_max_clusters(R, C, threads, smem, rows, hist);
    memo[key] = n;
    return n;
}

int memo_l2_clusters(int R, int C, int threads, size_t smem, bool hist = false)
{
    static std::mutex mu;
    static std::map<std::tuple<int, int, int, int, size_t, bool>, int> memo;
    int dev = 0;
    cudaGetDevice(&dev);
    const auto key = std::make_tuple(dev, R, C, threads, smem, hist);
    std::lock_guard<std::mutex> lock(mu);
    const auto it = memo.find(key);
    if (it != memo.end()) return it->second;
    const int n = l2_max_clusters(R, C, threads, smem, hist);
    if (n >= 0) memo[key] = n;       // errors (negative) are not kept
    return n;
}

// the run lengths to consider: the forced one, else RESIDENT_RUNS
std::vector<int> resident_runs(int forced)
{
    if (forced > 0) return {forced};
    return std::vector<int>(std::begin(RESIDENT_RUNS), std::end(RESIDENT_RUNS));
}

struct GridHost {
    empso_grid spec;
    GridDev dev;
    float *ex = nullptr, *ez = nullptr, *wavelet = nullptr, *Wx = nullptr, *Wz = nullptr;
    // irregular level grid (empso_set_levels)
    float *level_z = nullptr, *node_x = nullptr;
    int *level_off = nullptr;
    int4 *lidx = nullptr;
    float4 *lw = nullptr;
};

struct empso_ctx {
    int device = 0;
    int sm_count = 0;
    std::vector<GridHost> grids;
    GridDev *grids_dev = nullptr;
    float2 *rec_dev = nullptr;
    std::vector<float> rec_host;
    int nrec_total = 0;

    // workspace, grown on demand
    float *fields = nullptr;
    size_t fields_cap = 0;       // floats
    float *slots = nullptr;
    size_t slots_cap = 0;        // floats
    double *partial = nullptr;
    size_t partial_cap = 0;      // doubles
    unsigned char *stage_host = nullptr;  // pinned: instance table + shot weights
    unsigned char *stage_dev = nullptr;
    size_t stage_cap = 0;        // bytes
    cudaEvent_t stage_free = nullptr;
    int *counter = nullptr;

    // launch shape of the modelling kernel
    int kernel_kind = EMPSO_KERNEL_AUTO;
    int wave_threads = 512;
    int wave_ctas_per_sm = 1;
    size_t smem_optin = 0;          // max dynamic shared memory per block
    int forced_C = 0;               // 0: choose the cluster size, else use this one
    int forced_rows = 0;            // on-chip kernel: 0 choose the rows per thread, else use this many
    int last_path = 0;              // 1 streaming, 2 resident, 3 bulk-copy streaming (last launch)
    int last_C = 0;
    int last_rows = 0;              // on-chip launch: rows per thread
    int last_groups = 0;            // co-resident clusters (CTAs for the streaming kernels)
    int last_paired = 0;            // on-chip launch: units running two instances
    int *dev_err = nullptr;         // device status word set by bounded waits that give up
    unsigned long long *nonfinite = nullptr;  // non-finite misfits: {running, this call}
    bool strict = false;            // report non-finite misfits as EMPSO_NONFINITE

    // swarm
    bool has_pso = false;
    empso_pso pcfg{};
    PsoDev pso{};
    double *pso_mem = nullptr;
    int *pso_int = nullptr;

    // tuned (kind, cluster, rows per thread) choices by batch signature, and the cache file
    struct Tuned {
        int kind = 0, C = 0, rows = 0;
    };
    std::map<std::string, Tuned> tuned;
    std::string tune_cache;

    // captured generations (eval + EMPSO step), one per shape and buffers
    struct GraphEntry {
        std::string key;
        cudaGraphExec_t exec = nullptr;
        unsigned char *table = nullptr;
    };
    std::vector<GraphEntry> graphs;
    cudaStream_t cap_stream = nullptr;
    // the gradient's backward pass as independent chains of instances, each
    // on its own captured stream, so that one chain's memory waits and launch
    // gaps overlap another's work
    static constexpr int MAX_CHAINS = 8;
    int grad_chains = 0;            // 0: four chains from 16 instances up, else one
    cudaStream_t chain_stream[MAX_CHAINS - 1] = {};
    cudaEvent_t chain_fork = nullptr, chain_join[MAX_CHAINS - 1] = {};
    float *xf = nullptr;            // float copy of the swarm positions [P][D]
    double *gen_misfit = nullptr;   // misfit of the last captured generation [P]

    // surrogate network and the buffers of surrogate-assisted generations
    bool has_sur = false;
    SurDev sur;
    std::vector<void *> sur_mem;
    cudaStream_t sur_stream = nullptr;   // training of prescreen generations, beside the modelling
    cudaEvent_t sur_fork = nullptr, sur_done = nullptr;
    bool sur_done_rec = false;
    bool sur_overlap = false;            // train prescreen generations beside their modelling
    float sur_rho_min = 0.f;             // > 0: model the whole swarm after a pre-screened generation
                                         // whose rank correlation fell below this
    bool sur_screened = false;           // the last surrogate generation was pre-screened
    int sur_patience = 0;                // > 0: model the whole swarm after this many pre-screened
                                         // generations in a row without a new best misfit
    int sur_stall = 0;                   // such generations so far
    double sur_best = HUGE_VAL;          // best misfit when the count was last updated
    int *sel_rows = nullptr;        // [P] indices of the modelled particles
    float *xk = nullptr;            // [P][D] their positions
    double *fk = nullptr;           // [P] their misfits
    double *fit_full = nullptr;     // [P] fitness, +inf where not modelled
    double *rank_full = nullptr;    // [P] EM sort keys
    float *logphi = nullptr;        // [P] predictions

    // adjoint-state gradient workspace (grown on demand)
    struct AdjWork {
        float *a = nullptr, *B = nullptr, *H = nullptr, *mu = nullptr, *G = nullptr,
              *E = nullptr;
        size_t a_cap = 0, H_cap = 0, mu_cap = 0, E_cap = 0;   // floats
        AdjInst *insts = nullptr;
        size_t inst_cap = 0;
        double *phi = nullptr;
        size_t phi_cap = 0;
        std::string layout;       // grid and instance count the history was zeroed for
        float *fv = nullptr;      // FWI vectors: trial model, gradients [3][np]
        size_t fv_cap = 0;
        double *fd = nullptr;     // FWI reductions [8] and misfit [1]
        unsigned char *rtab = nullptr;   // on-chip forward pass: Inst [I], then work units [I]
        size_t rtab_cap = 0;
        int *counter = nullptr;          // its work queue
        size_t counter_cap = 0;
        float4 *slots = nullptr;         // L2 cluster forward pass: two time levels per cluster
        size_t slots_cap = 0;
        // forward + adjoint time loops captured once per grid, instance count
        // and instance table (their kernels read everything else from it)
        std::vector<std::pair<std::string, cudaGraphExec_t>> graphs;
    } adj;

    // kernel timing
    bool timing = false;
    bool timed = false;
    cudaEvent_t tev[4] = {nullptr, nullptr, nullptr, nullptr};

    std::string err;
};

namespace {

thread_local std::string g_create_error;

empso_status fail(empso_ctx *c, empso_status s, const std::string &msg)
{
    if (c) c->err = msg;
    else g_create_error = msg;
    return s;
}

#define CK(ctx, call)                                                                     \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? EMPSO_OOM : EMPSO_CUDA_ERROR, \
                        std::string(#call) + ": " + cudaGetErrorString(e_));              \
    } while (0)

}  // namespace

// Centred second-derivative weights of accuracy order 2R (Fornberg 1988).
bool empso::fd_weights(int order, double *c, int *R)
{
    static const double w2[] = {-2.0, 1.0};
    static const double w4[] = {-5.0 / 2.0, 4.0 / 3.0, -1.0 / 12.0};
    static const double w8[] = {-205.0 / 72.0, 8.0 / 5.0, -1.0 / 5.0, 8.0 / 315.0, -1.0 / 560.0};
    static const double w16[] = {-1077749.0 / 352800.0, 16.0 / 9.0, -14.0 / 45.0, 112.0 / 1485.0,
                                 -7.0 / 396.0, 112.0 / 32175.0, -2.0 / 3861.0, 16.0 / 315315.0,
                                 -1.0 / 411840.0};
    const double *w = nullptr;
    if (order == 2) { w = w2; *R = 1; }
    else if (order == 4) { w = w4; *R = 2; }
    else if (order == 8) { w = w8; *R = 4; }
    else if (order == 16) { w = w16; *R = 8; }
    else return false;
    for (int m = 0; m <= *R; ++m) c[m] = w[m];
    return true;
}

// Validation of a grid description and everything derived from it on the
// host: stencil weights, time axis (CFL rule unless dt is given), buffer
// layout.  Device table pointers stay null.
empso_status empso::derive_grid(const empso_grid &s, int id, GridDev &g, std::string &err)
{
    char buf[256];
    if (s.nx < 2 || s.nz < 2 || s.pad < 0 || !(s.hx > 0) || !(s.hz > 0) || !(s.t_rec > 0) ||
        !(s.f0 > 0) || !(s.vmax > 0) || !(s.vmin <= s.vmax) || s.kx < 2 || s.kz < 2 ||
        s.kx > 64 || s.kz > 64 || (s.interp_mode != 0 && s.interp_mode != 1)) {
        snprintf(buf, sizeof buf, "grid %d: invalid sizes/spacings/bounds (need nx,nz>=2, "
                 "pad>=0, h>0, T>0, f0>0, vmin<=vmax, 2<=kx,kz<=64, mode 0|1)", id);
        err = buf;
        return EMPSO_INVALID_ARG;
    }
    double c[MAX_R + 1];
    int R = 0;
    if (!fd_weights(s.space_order, c, &R)) {
        snprintf(buf, sizeof buf, "grid %d: space order %d not in {2,4,8,16}", id, s.space_order);
        err = buf;
        return EMPSO_UNSUPPORTED;
    }
    memset(&g, 0, sizeof g);
    g.nx = s.nx;
    g.nz = s.nz;
    g.pad = s.pad;
    g.R = R;
    g.NX = s.nx + 2 * s.pad;
    g.NZ = s.nz + 2 * s.pad;
    g.NQ = (g.NX + 3) / 4;
    g.pitch = ((4 * g.NQ + 2 * HALO) + 31) / 32 * 32;
    g.rows = g.NZ + 2 * HALO;
    g.field = (long long)g.rows * g.pitch;
    g.kx = s.kx;
    g.kz = s.kz;
    g.K = s.kx * s.kz;
    g.mode = s.interp_mode;
    g.hx = s.hx;
    g.hz = s.hz;
    g.vmin = s.vmin;
    g.vmax = s.vmax;
    // time axis: dt = T / (nt - 1), nt = ceil(T / (0.9 dt_cfl)) + 1 unless given
    double dt = s.dt, T = s.t_rec;
    int nt;
    if (dt <= 0) {
        double rho = c[0];
        for (int m = 1; m <= R; ++m) rho += 2.0 * ((m & 1) ? -c[m] : c[m]);
        rho = std::fabs(rho);
        const double hx = s.hx, hz = s.hz;
        const double dtmax = 2.0 / (s.vmax * std::sqrt(rho * (1.0 / (hx * hx) + 1.0 / (hz * hz))));
        nt = (int)std::ceil(T / (0.9 * dtmax)) + 1;
        dt = T / (double)(nt - 1);
    } else {
        nt = (int)std::lround(T / dt) + 1;
    }
    if (nt < 2 || nt > (1 << 24)) {
        snprintf(buf, sizeof buf, "grid %d: %d time steps out of range", id, nt);
        err = buf;
        return EMPSO_INVALID_ARG;
    }
    g.nt = nt;
    g.dt = (float)dt;
    const double ihx2 = 1.0 / ((double)s.hx * s.hx), ihz2 = 1.0 / ((double)s.hz * s.hz);
    for (int m = 0; m <= MAX_R; ++m) {
        const double cm = m <= R ? c[m] : 0.0;
        g.c[m] = (float)cm;
        g.cxm[m] = (float)(cm * ihx2);
        g.czm[m] = (float)(cm * ihz2);
    }
    g.cxm[0] = (float)(c[0] * (ihx2 + ihz2));
    g.czm[0] = 0.f;
    double cres = c[0];
    for (int m = 1; m <= std::min(R, 2); ++m) cres += 2.0 * c[m];
    g.cres = (float)(cres * (ihx2 + ihz2));
    return EMPSO_OK;
}

namespace {

empso_status setup_grid(empso_ctx *ctx, GridHost &G, int id)
{
    const empso_grid &s = G.spec;
    GridDev &g = G.dev;
    std::string err;
    const empso_status rc = derive_grid(s, id, g, err);
    if (rc != EMPSO_OK) return fail(ctx, rc, err);
    const int nt = g.nt;
    CK(ctx, cudaMalloc(&G.ex, sizeof(float) * g.pitch));
    CK(ctx, cudaMalloc(&G.ez, sizeof(float) * g.rows));
    CK(ctx, cudaMalloc(&G.wavelet, sizeof(float) * nt));
    CK(ctx, cudaMalloc(&G.Wx, sizeof(float) * s.nx * s.kx));
    CK(ctx, cudaMalloc(&G.Wz, sizeof(float) * s.nz * s.kz));
    g.ex = G.ex;
    g.ez = G.ez;
    g.wavelet = G.wavelet;
    g.Wx = G.Wx;
    g.Wz = G.Wz;
    CK(ctx, launch_grid_tables(g, G.ex, G.ez, G.wavelet, G.Wx, G.Wz, s.vmax, s.f0, 0));
    return EMPSO_OK;
}

empso_status grow(empso_ctx *ctx, void **p, size_t *cap, size_t need_bytes, size_t elem)
{
    if (need_bytes <= *cap * elem) return EMPSO_OK;
    if (*p) {
        CK(ctx, cudaDeviceSynchronize());
        CK(ctx, cudaFree(*p));
        *p = nullptr;
        *cap = 0;
    }
    size_t bytes = need_bytes + need_bytes / 8;
    CK(ctx, cudaMalloc(p, bytes));
    *cap = bytes / elem;
    return EMPSO_OK;
}

empso_status grow_stage(empso_ctx *ctx, size_t bytes)
{
    if (bytes <= ctx->stage_cap) return EMPSO_OK;
    CK(ctx, cudaEventSynchronize(ctx->stage_free));
    if (ctx->stage_host) cudaFreeHost(ctx->stage_host);
    if (ctx->stage_dev) {
        CK(ctx, cudaDeviceSynchronize());
        cudaFree(ctx->stage_dev);
    }
    ctx->stage_host = nullptr;
    ctx->stage_dev = nullptr;
    size_t cap = std::max<size_t>(bytes * 2, 1 << 16);
    CK(ctx, cudaMallocHost(&ctx->stage_host, cap));
    CK(ctx, cudaMalloc(&ctx->stage_dev, cap));
    ctx->stage_cap = cap;
    return EMPSO_OK;
}

// Validate shots against the grids and the receiver table.
empso_status check_shots(empso_ctx *ctx, const empso_shot *shots, int S, int only_grid)
{
    if (!shots || S <= 0) return fail(ctx, EMPSO_INVALID_ARG, "need at least one shot");
    char buf[256];
    for (int s = 0; s < S; ++s) {
        const empso_shot &sh = shots[s];
        if (sh.grid_id < 0 || sh.grid_id >= (int)ctx->grids.size()) {
            snprintf(buf, sizeof buf, "shot %d: grid_id %d out of range", s, sh.grid_id);
            return fail(ctx, EMPSO_INVALID_ARG, buf);
        }
        if (only_grid >= 0 && sh.grid_id != only_grid) {
            snprintf(buf, sizeof buf, "shot %d: gridded models need every shot on one grid", s);
            return fail(ctx, EMPSO_INVALID_ARG, buf);
        }
        const empso_grid &g = ctx->grids[sh.grid_id].spec;
        const float Lx = (g.nx - 1) * g.hx, Lz = (g.nz - 1) * g.hz;
        if (!(sh.sx >= 0 && sh.sx <= Lx && sh.sz >= 0 && sh.sz <= Lz)) {
            snprintf(buf, sizeof buf, "shot %d: source (%g, %g) outside the %g x %g m domain", s,
                     sh.sx, sh.sz, Lx, Lz);
            return fail(ctx, EMPSO_INVALID_ARG, buf);
        }
        if (sh.nrec < 0 || sh.rec_begin < 0 || sh.rec_begin + (long long)sh.nrec > ctx->nrec_total) {
            snprintf(buf, sizeof buf, "shot %d: receivers [%d, %d) outside the table of %d", s,
                     sh.rec_begin, sh.rec_begin + sh.nrec, ctx->nrec_total);
            return fail(ctx, EMPSO_INVALID_ARG, buf);
        }
        for (int r = sh.rec_begin; r < sh.rec_begin + sh.nrec; ++r) {
            const float x = ctx->rec_host[2 * r], z = ctx->rec_host[2 * r + 1];
            if (!(x >= 0 && x <= Lx && z >= 0 && z <= Lz)) {
                snprintf(buf, sizeof buf, "shot %d: receiver %d at (%g, %g) outside its grid", s, r,
                         x, z);
                return fail(ctx, EMPSO_INVALID_ARG, buf);
            }
        }
        if (!std::isfinite(sh.weight)) {
            snprintf(buf, sizeof buf, "shot %d: non-finite weight", s);
            return fail(ctx, EMPSO_INVALID_ARG, buf);
        }
    }
    return EMPSO_OK;
}

// Model source for a batch: control-node particles or gridded velocities.
struct Models {
    const float *particles = nullptr;  // [M][K]
    const float *vel = nullptr;        // [M][nz][nx]
    int M = 0;
};

// Everything the host decides about one persistent modelling launch.
// Instances of the L2-resident cluster kernel in flight are capped so that
// their time levels and model fields fit this share of the 129 MB L2.
constexpr long long L2_BUDGET_BYTES = 96LL << 20;

struct Plan {
    int M = 0, S = 0;
    long long n_inst = 0, maxfield = 0;
    std::vector<long long> fbase;      // per grid: offset of its M model fields, -1 if unused
    bool resident = false;
    int resR = 0, resC = 0, res_threads = 0, res_clusters = 0, res_rows = 0, ring_pitch = 0;
    size_t res_smem = 0;
    std::vector<char> res_pair;        // per grid: two instances share a cluster (half each)
    std::vector<int> res_run;          // per grid: rows per run of its instances (0: res_rows)
    const int4 *units = nullptr;       // device work units of the on-chip kernel
    int n_units = 0, n_paired = 0;
    int n_ctas = 0;
    bool l2 = false;                   // L2-resident cluster kernel
    int l2C = 0, l2_clusters = 0, l2_threads = 0;
    long long l2_slot_f4 = 0;
    size_t l2_smem = 0;
    bool stream_tma = false;           // streaming path: row-pipelined bulk-copy kernel
    int st_threads = 0, st_R = 0, rec_max = 0;
    size_t st_smem = 0;
    const Inst *insts = nullptr;       // device instance table
    const float *weights = nullptr;    // device shot weights
};

// Signature of a batch for the tuned-choice table: the grids its shots use
// (with their sizes and orders), their shot counts, and the model count.
std::string batch_key(const empso_ctx *ctx, const empso_shot *shots, int S, int M)
{
    std::vector<int> count(ctx->grids.size(), 0);
    for (int s = 0; s < S; ++s) ++count[shots[s].grid_id];
    std::string k = "M" + std::to_string(M);
    for (size_t g = 0; g < count.size(); ++g) {
        if (!count[g]) continue;
        const GridDev &d = ctx->grids[g].dev;
        k += "|" + std::to_string(d.NX) + "x" + std::to_string(d.NZ) + "o" + std::to_string(2 * d.R) +
             "t" + std::to_string(d.nt) + "s" + std::to_string(count[g]);
    }
    return k;
}

// Choose the kernel, size the workspace and build the instance table.  With
// `table` the table is copied synchronously into that device buffer (graph
// capture); otherwise it goes through the pinned staging buffer on `st`.
empso_status plan_batch(empso_ctx *ctx, const Models &mod, const empso_shot *shots, int S,
                        const float *d_obs, float *traces, Plan &p, unsigned char *table,
                        cudaStream_t st)
{
    const int M = mod.M;
    const int ng = (int)ctx->grids.size();
    p.M = M;
    p.S = S;
    std::vector<long long> doff(S + 1, 0);
    for (int s = 0; s < S; ++s)
        doff[s + 1] = doff[s] + (long long)ctx->grids[shots[s].grid_id].dev.nt * shots[s].nrec;
    p.fbase.assign(ng, -1);
    long long ftotal = 0;
    p.maxfield = 0;
    for (int s = 0; s < S; ++s) {
        const int gid = shots[s].grid_id;
        if (p.fbase[gid] < 0) {
            p.fbase[gid] = ftotal;
            ftotal += (long long)M * ctx->grids[gid].dev.field;
            p.maxfield = std::max(p.maxfield, ctx->grids[gid].dev.field);
        }
    }
    p.n_inst = (long long)M * S;
    if (p.n_inst > (1LL << 30)) return fail(ctx, EMPSO_INVALID_ARG, "too many instances");
    empso_status rc;

    // kernel and cluster size: explicit settings, else the tuned choice, else
    // the on-chip kernel with the cluster size that keeps the most SMs busy
    int kind = ctx->kernel_kind, forcedC = ctx->forced_C, forcedRows = ctx->forced_rows;
    if (forcedC == 0 && forcedRows == 0) {
        auto it = ctx->tuned.find(batch_key(ctx, shots, S, M));
        if (it != ctx->tuned.end() && (kind == EMPSO_KERNEL_AUTO || kind == it->second.kind)) {
            kind = it->second.kind;
            forcedC = it->second.C;
            forcedRows = it->second.rows;
        }
    }
    int resR = -1;
    for (int gid = 0; gid < ng; ++gid) {   // one stencil radius per on-chip launch
        if (p.fbase[gid] < 0) continue;
        const int R = ctx->grids[gid].dev.R;
        resR = (resR < 0 || resR == R) ? R : 0;
    }
    // the cluster and bulk-copy kernels hold stencils up to radius 4; order
    // 16 (and mixed orders) run on the plain streaming kernel
    if (resR > MAX_R_FAST) resR = 0;
    p.resident = false;
    if ((kind == EMPSO_KERNEL_AUTO || kind == EMPSO_KERNEL_RESIDENT) && resR > 0) {
        long long best_sms = 0;
        int nrec_max = 0;
        for (int s = 0; s < S; ++s) nrec_max = std::max(nrec_max, (int)shots[s].nrec);
        const int ring_pitch = nrec_max;
        // every cluster size and rows-per-thread shape; the most SMs busy wins,
        // the longer runs (fewer, fatter threads) on a tie
        for (int C = 1; C <= 16; ++C)
            for (const int rows : resident_runs(forcedRows)) {
            if (forcedC > 0 && C != forcedC) continue;
            bool ok = true;
            size_t sm = 0;
            int threads = 32;
            for (int gid = 0; gid < ng && ok; ++gid) {
                if (p.fbase[gid] < 0) continue;
                const GridDev &g = ctx->grids[gid].dev;
                ok = resident_fits(g, C, ring_pitch, ctx->smem_optin, rows);
                sm = std::max(sm, resident_smem_bytes(g, C, ring_pitch));
                threads = std::max(threads, resident_threads(g, C, rows));
            }
            if (!ok) continue;
            // a grid runs two instances per cluster, one on each half, when it
            // fits C / 2 CTAs without raising the launch's shared memory or threads
            std::vector<char> pair(ng, 0);
            if (C % 2 == 0)
                for (int gid = 0; gid < ng; ++gid) {
                    if (p.fbase[gid] < 0) continue;
                    const GridDev &g = ctx->grids[gid].dev;
                    pair[gid] = resident_fits(g, C / 2, ring_pitch, ctx->smem_optin, rows) &&
                                resident_smem_bytes(g, C / 2, ring_pitch) <= sm &&
                                resident_threads(g, C / 2, rows) <= threads;
                }
            const int nc = (int)std::min<long long>(memo_resident_clusters(resR, C, threads, sm, rows), p.n_inst);
            const long long sms = (long long)nc * C;
            if (nc > 0 && sms > best_sms) {
                best_sms = sms;
                p.resident = true;
                p.res_pair = pair;
                p.resR = resR;
                p.resC = C;
                p.res_rows = rows;
                p.res_smem = sm;
                p.res_threads = threads;
                p.res_clusters = nc;
                p.ring_pitch = ring_pitch;
            }
        }
    }
    if (kind == EMPSO_KERNEL_RESIDENT && !p.resident)
        return fail(ctx, EMPSO_UNSUPPORTED,
                    "the batch does not fit the on-chip kernel (grid too large or mixed orders)");
    // a grid whose work items fill few of the launch's threads (the smaller
    // grid of an uneven batch) runs shorter runs, more per column
    p.res_run.assign(ng, 0);
    if (p.resident)
        for (int gid = 0; gid < ng; ++gid)
            if (p.fbase[gid] >= 0)
                p.res_run[gid] = resident_grid_run(ctx->grids[gid].dev, p.res_pair[gid] ? p.resC / 2 : p.resC,
                                                   p.res_threads, p.res_rows);
    // L2-resident cluster kernel for grids the on-chip kernel cannot hold:
    // the cluster size that keeps the most SMs busy while every instance in
    // flight (two time levels and the model field) stays within the L2 budget
    p.l2 = false;
    if (!p.resident && resR > 0 && (kind == EMPSO_KERNEL_AUTO || kind == EMPSO_KERNEL_CLUSTER_L2)) {
        int nrec_max = 0;
        for (int s = 0; s < S; ++s) nrec_max = std::max(nrec_max, (int)shots[s].nrec);
        const size_t sm = l2_smem_bytes(nrec_max);
        long long best_sms = 0;
        for (int C : {16, 12, 10, 8, 6, 4, 3, 2, 1}) {
            if (forcedC > 0 && C != forcedC) continue;
            bool ok = sm <= ctx->smem_optin;
            long long slot = 0, inst_bytes = 0, items = 32;
            for (int gid = 0; gid < ng && ok; ++gid) {
                if (p.fbase[gid] < 0) continue;
                const GridDev &g = ctx->grids[gid].dev;
                ok = l2_fits(g, C);
                slot = std::max(slot, l2_slot_f4(g, C));
                inst_bytes = std::max(inst_bytes, 32 * l2_slot_f4(g, C) + 4 * g.field);
                const int rows_c = (g.NZ + C - 1) / C;
                items = std::max<long long>(items, (long long)g.NQ * ((rows_c + 7) / 8));
            }
            if (!ok) continue;
            const int threads = (int)std::min<long long>(l2_max_threads(), (items + 31) / 32 * 32);
            CK(ctx, l2_configure(resR, sm, C));
            const long long by_l2 = std::max<long long>(1, L2_BUDGET_BYTES / std::max<long long>(inst_bytes, 1));
            const int occ = memo_l2_clusters(resR, C, threads, sm);
            if (occ < 0)
                return fail(ctx, EMPSO_CUDA_ERROR,
                            std::string("L2 cluster kernel occupancy (C = ") + std::to_string(C) +
                                "): " + cudaGetErrorString((cudaError_t)(-occ)));
            const int nc = (int)std::min<long long>(std::min<long long>(occ, p.n_inst), by_l2);
            const long long sms = (long long)nc * C;
            if (nc > 0 && sms > best_sms) {
                best_sms = sms;
                p.l2 = true;
                p.resR = resR;
                p.l2C = C;
                p.l2_clusters = nc;
                p.l2_threads = threads;
                p.l2_slot_f4 = slot;
                p.l2_smem = sm;
                p.ring_pitch = nrec_max;
            }
        }
    }
    if (kind == EMPSO_KERNEL_CLUSTER_L2 && !p.l2)
        return fail(ctx, EMPSO_UNSUPPORTED, "the batch does not fit the L2 cluster kernel");
    int max_ctas = ctx->sm_count * ctx->wave_ctas_per_sm;
    if (!p.resident && !p.l2 && resR > 0) {
        // row-pipelined streaming kernel: one thread per float4 column group
        int nq = 0, pitch = 0, nrec_max = 0;
        for (int gid = 0; gid < ng; ++gid) {
            if (p.fbase[gid] < 0) continue;
            nq = std::max(nq, ctx->grids[gid].dev.NQ);
            pitch = std::max(pitch, ctx->grids[gid].dev.pitch);
        }
        for (int s = 0; s < S; ++s) nrec_max = std::max(nrec_max, (int)shots[s].nrec);
        const size_t sm = stream_smem_bytes(resR, pitch, nrec_max);
        if (nq <= stream_max_threads() && sm <= ctx->smem_optin) {
            p.stream_tma = true;
            p.st_R = resR;
            p.st_threads = std::max(64, (nq + 31) / 32 * 32);
            p.st_smem = sm;
            p.rec_max = nrec_max;
            // shared memory decides how many of these CTAs share an SM
            const int per_sm = std::max(1, (int)(ctx->smem_optin / std::max<size_t>(sm, 1)));
            max_ctas = ctx->sm_count * std::min(per_sm, 2);
        }
    }
    p.n_ctas = (int)std::min<long long>(p.n_inst, max_ctas);
    if ((rc = grow(ctx, (void **)&ctx->fields, &ctx->fields_cap, sizeof(float) * ftotal,
                   sizeof(float))) != EMPSO_OK)
        return rc;
    if (p.l2 &&
        (rc = grow(ctx, (void **)&ctx->slots, &ctx->slots_cap,
                   sizeof(float4) * 2 * (size_t)p.l2_slot_f4 * p.l2_clusters, sizeof(float))) != EMPSO_OK)
        return rc;
    if (!p.resident && !p.l2 &&
        (rc = grow(ctx, (void **)&ctx->slots, &ctx->slots_cap,
                   sizeof(float) * 2 * p.maxfield * p.n_ctas, sizeof(float))) != EMPSO_OK)
        return rc;
    if ((rc = grow(ctx, (void **)&ctx->partial, &ctx->partial_cap, sizeof(double) * p.n_inst,
                   sizeof(double))) != EMPSO_OK)
        return rc;
    const size_t inst_bytes = sizeof(Inst) * p.n_inst;
    const size_t wofs = (inst_bytes + 255) / 256 * 256;
    const size_t uofs = wofs + (sizeof(float) * S + 15) / 16 * 16;
    const size_t tbytes = uofs + sizeof(int4) * p.n_inst;
    if ((rc = grow_stage(ctx, tbytes)) != EMPSO_OK) return rc;

    // instance table, longest work first so the dynamic queue balances
    std::vector<long long> order(p.n_inst);
    for (long long q = 0; q < p.n_inst; ++q) order[q] = q;
    auto work = [&](long long q) {
        const GridDev &g = ctx->grids[shots[q % S].grid_id].dev;
        return (double)g.field * g.nt;
    };
    std::stable_sort(order.begin(), order.end(),
                     [&](long long a, long long b) { return work(a) > work(b); });
    CK(ctx, cudaEventSynchronize(ctx->stage_free));  // previous upload has left the buffer
    Inst *hi = reinterpret_cast<Inst *>(ctx->stage_host);
    const long long per_model = doff[S];
    for (long long k = 0; k < p.n_inst; ++k) {
        const long long q = order[k];
        const int m = (int)(q / S), s = (int)(q % S);
        const empso_shot &sh = shots[s];
        const GridDev &g = ctx->grids[sh.grid_id].dev;
        Inst in{};
        in.a = ctx->fields + p.fbase[sh.grid_id] + (long long)m * g.field;
        in.dobs = d_obs ? d_obs + doff[s] : nullptr;
        in.traces = traces ? traces + (long long)m * per_model + doff[s] : nullptr;
        in.rec = ctx->rec_dev + sh.rec_begin;
        in.grid = sh.grid_id;
        in.nrec = sh.nrec;
        in.sx = sh.sx;
        in.sz = sh.sz;
        in.out = (int)q;
        in.run = p.resident ? p.res_run[sh.grid_id] : 0;
        hi[k] = in;
    }
    float *wh = reinterpret_cast<float *>(ctx->stage_host + wofs);
    for (int s = 0; s < S; ++s) wh[s] = shots[s].weight;
    // work units of the on-chip kernel: consecutive instances of a paired grid
    // (the sort keeps a grid's instances together) share a cluster
    int4 *uh = reinterpret_cast<int4 *>(ctx->stage_host + uofs);
    p.n_units = 0;
    p.n_paired = 0;
    for (long long k = 0; k < p.n_inst;) {
        const int gid = shots[order[k] % S].grid_id;
        if (p.resident && p.res_pair[gid] && k + 1 < p.n_inst && shots[order[k + 1] % S].grid_id == gid) {
            uh[p.n_units++] = make_int4((int)k, (int)k + 1, 1, 0);
            ++p.n_paired;
            k += 2;
        } else {
            uh[p.n_units++] = make_int4((int)k, -1, 0, 0);
            k += 1;
        }
    }
    unsigned char *dst = table ? table : ctx->stage_dev;
    if (table) {
        CK(ctx, cudaMemcpy(table, ctx->stage_host, tbytes, cudaMemcpyHostToDevice));
    } else {
        CK(ctx, cudaMemcpyAsync(ctx->stage_dev, ctx->stage_host, tbytes, cudaMemcpyHostToDevice, st));
        CK(ctx, cudaEventRecord(ctx->stage_free, st));
    }
    p.insts = reinterpret_cast<const Inst *>(dst);
    p.weights = reinterpret_cast<const float *>(dst + wofs);
    p.units = reinterpret_cast<const int4 *>(dst + uofs);
    return EMPSO_OK;
}

size_t table_bytes(long long n_inst, int S)
{
    return (sizeof(Inst) * n_inst + 255) / 256 * 256 + (sizeof(float) * S + 15) / 16 * 16 +
           sizeof(int4) * n_inst;
}

// Timing event on `st`; inside a stream capture it becomes an event-record
// node that records whenever the graph runs.
cudaError_t mark(cudaEvent_t ev, cudaStream_t st)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(st, &cs);
    if (e != cudaSuccess) return e;
    if (cs == cudaStreamCaptureStatusActive) return cudaEventRecordWithFlags(ev, st, cudaEventRecordExternal);
    return cudaEventRecord(ev, st);
}

// Enqueue the planned launch: model fields, queue reset, persistent
// modelling kernel, misfit reduction (when `misfit` is given).
empso_status enqueue_batch(empso_ctx *ctx, const Models &mod, const Plan &p, double *misfit,
                           cudaStream_t st, cudaEvent_t before_model = nullptr)
{
    const int ng = (int)ctx->grids.size();
    if (ctx->timing) CK(ctx, mark(ctx->tev[0], st));
    for (int gid = 0; gid < ng; ++gid) {
        if (p.fbase[gid] < 0) continue;
        const GridDev &g = ctx->grids[gid].dev;
        float *dst = ctx->fields + p.fbase[gid];
        if (mod.particles) CK(ctx, launch_interp(g, mod.particles, p.M, dst, g.field, nullptr, st));
        else CK(ctx, launch_vel_to_field(g, mod.vel, p.M, dst, g.field, st));
    }
    CK(ctx, cudaMemsetAsync(ctx->counter, 0, sizeof(int), st));
    if (ctx->timing) CK(ctx, mark(ctx->tev[1], st));
    if (before_model) CK(ctx, cudaEventRecord(before_model, st));
    if (p.resident) {
        // the variant for several grids: paired units, or a grid with its own run length
        const bool multi = p.n_paired > 0 || std::any_of(p.res_run.begin(), p.res_run.end(), [](int r) { return r > 0; });
        CK(ctx, launch_wave_resident(p.resR, ctx->grids_dev, p.insts, p.units, p.n_units, multi,
                                     ctx->counter, p.resC, p.res_clusters, p.res_threads, p.res_rows,
                                     p.ring_pitch, p.res_smem, ctx->partial, st));
        ctx->last_path = 2;
        ctx->last_C = p.resC;
        ctx->last_rows = p.res_rows;
        ctx->last_groups = p.res_clusters;
        ctx->last_paired = p.n_paired;
    } else if (p.l2) {
        CK(ctx, launch_wave_l2(p.resR, ctx->grids_dev, p.insts,
                               (int)p.n_inst, ctx->counter, p.l2C, p.l2_clusters, p.l2_threads,
                               reinterpret_cast<float4 *>(ctx->slots), p.l2_slot_f4, p.ring_pitch,
                               p.l2_smem, ctx->partial, st));
        ctx->last_path = 4;
        ctx->last_C = p.l2C;
        ctx->last_groups = p.l2_clusters;
    } else if (p.stream_tma) {
        CK(ctx, launch_wave_stream(p.st_R, ctx->grids_dev, p.insts, (int)p.n_inst, ctx->counter,
                                   ctx->slots, 2 * p.maxfield, p.n_ctas, p.st_threads, p.st_smem,
                                   p.rec_max, ctx->dev_err, ctx->partial, st));
        ctx->last_path = 3;
        ctx->last_C = 1;
        ctx->last_groups = p.n_ctas;
    } else {
        CK(ctx, launch_wave(ctx->grids_dev, p.insts, (int)p.n_inst, ctx->counter, ctx->slots,
                            2 * p.maxfield, p.n_ctas, ctx->wave_threads, ctx->partial, st));
        ctx->last_path = 1;
        ctx->last_C = 1;
        ctx->last_groups = p.n_ctas;
    }
    if (ctx->timing) CK(ctx, mark(ctx->tev[2], st));
    if (misfit)
        CK(ctx, launch_finalize(ctx->partial, p.weights, p.M, p.S, misfit, ctx->nonfinite, st));
    if (ctx->timing) {
        CK(ctx, mark(ctx->tev[3], st));
        ctx->timed = true;
    }
    return EMPSO_OK;
}

empso_status run_batch(empso_ctx *ctx, const Models &mod, const empso_shot *shots, int S,
                       const float *d_obs, float *traces, double *misfit, cudaStream_t st,
                       cudaEvent_t before_model = nullptr)
{
    Plan p;
    empso_status rc = plan_batch(ctx, mod, shots, S, d_obs, traces, p, nullptr, st);
    if (rc) return rc;
    return enqueue_batch(ctx, mod, p, misfit, st, before_model);
}

// Strict mode: zero the per-call count of non-finite misfits before the
// work, read it back (synchronising the stream) after it.
empso_status strict_begin(empso_ctx *ctx, cudaStream_t st)
{
    if (ctx->strict) CK(ctx, cudaMemsetAsync(ctx->nonfinite + 1, 0, sizeof(unsigned long long), st));
    return EMPSO_OK;
}

empso_status strict_end(empso_ctx *ctx, empso_status rc, cudaStream_t st)
{
    if (rc || !ctx->strict) return rc;
    unsigned long long n = 0;
    CK(ctx, cudaMemcpyAsync(&n, ctx->nonfinite + 1, sizeof n, cudaMemcpyDeviceToHost, st));
    CK(ctx, cudaStreamSynchronize(st));
    if (n)
        return fail(ctx, EMPSO_NONFINITE,
                    std::to_string(n) + " non-finite misfit(s), returned as +inf");
    return EMPSO_OK;
}

// Re-upload one grid's device record after a change of its parameterisation
// and drop the captured generations (their interpolation launches hold the
// old record by value).
empso_status grid_changed(empso_ctx *ctx, int gid)
{
    CK(ctx, cudaDeviceSynchronize());
    CK(ctx, cudaMemcpy(ctx->grids_dev + gid, &ctx->grids[gid].dev, sizeof(GridDev),
                       cudaMemcpyHostToDevice));
    for (auto &e : ctx->graphs) {
        if (e.exec) cudaGraphExecDestroy(e.exec);
        cudaFree(e.table);
    }
    ctx->graphs.clear();
    for (auto &e : ctx->adj.graphs)
        if (e.second) cudaGraphExecDestroy(e.second);
    ctx->adj.graphs.clear();
    return EMPSO_OK;
}

void free_ctx(empso_ctx *c)
{
    if (!c) return;
    cudaDeviceSynchronize();
    for (auto &G : c->grids) {
        cudaFree(G.ex);
        cudaFree(G.ez);
        cudaFree(G.wavelet);
        cudaFree(G.Wx);
        cudaFree(G.Wz);
        cudaFree(G.level_z);
        cudaFree(G.node_x);
        cudaFree(G.level_off);
        cudaFree(G.lidx);
        cudaFree(G.lw);
    }
    cudaFree(c->grids_dev);
    cudaFree(c->rec_dev);
    cudaFree(c->fields);
    cudaFree(c->slots);
    cudaFree(c->partial);
    cudaFree(c->stage_dev);
    cudaFree(c->counter);
    cudaFree(c->dev_err);
    cudaFree(c->nonfinite);
    cudaFree(c->adj.a);       // B lies inside a; G and J inside mu
    cudaFree(c->adj.H);
    cudaFree(c->adj.mu);
    cudaFree(c->adj.E);
    cudaFree(c->adj.insts);
    cudaFree(c->adj.phi);
    cudaFree(c->adj.fv);
    for (auto &e : c->adj.graphs)
        if (e.second) cudaGraphExecDestroy(e.second);
    cudaFree(c->adj.fd);
    cudaFree(c->adj.rtab);
    cudaFree(c->adj.counter);
    cudaFree(c->adj.slots);
    cudaFree(c->pso_mem);
    cudaFree(c->pso_int);
    cudaFree(c->xf);
    cudaFree(c->gen_misfit);
    for (auto &e : c->graphs) {
        if (e.exec) cudaGraphExecDestroy(e.exec);
        cudaFree(e.table);
    }
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    for (int i = 0; i < empso_ctx::MAX_CHAINS - 1; ++i) {
        if (c->chain_stream[i]) cudaStreamDestroy(c->chain_stream[i]);
        if (c->chain_join[i]) cudaEventDestroy(c->chain_join[i]);
    }
    if (c->chain_fork) cudaEventDestroy(c->chain_fork);
    for (void *p : c->sur_mem) cudaFree(p);
    if (c->sur_stream) cudaStreamDestroy(c->sur_stream);
    if (c->sur_fork) cudaEventDestroy(c->sur_fork);
    if (c->sur_done) cudaEventDestroy(c->sur_done);
    if (c->stage_host) cudaFreeHost(c->stage_host);
    if (c->stage_free) cudaEventDestroy(c->stage_free);
    for (auto &e : c->tev)
        if (e) cudaEventDestroy(e);
    delete c;
}

}  // namespace

void empso::set_global_error(const char *msg) { g_create_error = msg; }

extern "C" {

const char *empso_status_string(empso_status s)
{
    switch (s) {
    case EMPSO_OK: return "ok";
    case EMPSO_INVALID_ARG: return "invalid argument";
    case EMPSO_OOM: return "out of memory";
    case EMPSO_CUDA_ERROR: return "CUDA error";
    case EMPSO_NONFINITE: return "non-finite misfit";
    case EMPSO_TIMEOUT: return "device wait timed out";
    case EMPSO_UNSUPPORTED: return "unsupported";
    case EMPSO_NOT_INITIALIZED: return "not initialised";
    case EMPSO_IO_ERROR: return "file error";
    default: return "unknown status";
    }
}

const char *empso_last_error(const empso_ctx *ctx)
{
    return ctx ? ctx->err.c_str() : g_create_error.c_str();
}

empso_status empso_create(const empso_grid *grids, int32_t ngrids, const float *rec_xz,
                          int32_t nrec_total, const empso_pso *pso, const double *xmin,
                          const double *xmax, empso_ctx **out)
{
    g_create_error.clear();
    if (!out) return fail(nullptr, EMPSO_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!grids || ngrids <= 0 || ngrids > 64)
        return fail(nullptr, EMPSO_INVALID_ARG, "need 1..64 grids");
    if (nrec_total < 0 || (nrec_total > 0 && !rec_xz))
        return fail(nullptr, EMPSO_INVALID_ARG, "bad receiver table");
    empso_ctx *ctx = new (std::nothrow) empso_ctx();
    if (!ctx) return fail(nullptr, EMPSO_OOM, "host allocation failed");
    auto bail = [&](empso_status s) {
        g_create_error = ctx->err;
        free_ctx(ctx);
        return s;
    };
    if (cudaGetDevice(&ctx->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, ctx->device) !=
            cudaSuccess) {
        ctx->err = "no CUDA device";
        return bail(EMPSO_CUDA_ERROR);
    }
    empso_status rc;
    ctx->grids.resize(ngrids);
    for (int i = 0; i < ngrids; ++i) {
        ctx->grids[i].spec = grids[i];
        if ((rc = setup_grid(ctx, ctx->grids[i], i)) != EMPSO_OK) return bail(rc);
    }
    auto ck = [&](cudaError_t e, const char *what) {
        if (e == cudaSuccess) return EMPSO_OK;
        ctx->err = std::string(what) + ": " + cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? EMPSO_OOM : EMPSO_CUDA_ERROR;
    };
    ctx->nrec_total = nrec_total;
    ctx->rec_host.assign(rec_xz, rec_xz + 2 * (size_t)nrec_total);
    if ((rc = ck(cudaMalloc(&ctx->rec_dev, sizeof(float2) * std::max(1, nrec_total)), "receivers")))
        return bail(rc);
    if (nrec_total > 0 &&
        (rc = ck(cudaMemcpy(ctx->rec_dev, rec_xz, sizeof(float2) * nrec_total,
                            cudaMemcpyHostToDevice), "receiver copy")))
        return bail(rc);
    std::vector<GridDev> gd(ngrids);
    for (int i = 0; i < ngrids; ++i) gd[i] = ctx->grids[i].dev;
    if ((rc = ck(cudaMalloc(&ctx->grids_dev, sizeof(GridDev) * ngrids), "grid table")) ||
        (rc = ck(cudaMemcpy(ctx->grids_dev, gd.data(), sizeof(GridDev) * ngrids,
                            cudaMemcpyHostToDevice), "grid table copy")))
        return bail(rc);
    if ((rc = ck(cudaMalloc(&ctx->counter, sizeof(int)), "counter")) ||
        (rc = ck(cudaEventCreateWithFlags(&ctx->stage_free, cudaEventDisableTiming), "event")))
        return bail(rc);
    ctx->wave_ctas_per_sm = std::max(1, wave_max_ctas_per_sm(ctx->wave_threads));
    {
        int optin = 0;
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device);
        // keep room for the kernel's static shared memory
        ctx->smem_optin = optin > 1024 ? (size_t)optin - 1024 : 0;
        for (int R : {1, 2, 4}) {
            if ((rc = ck(resident_configure(R, ctx->smem_optin, 16), "on-chip kernel attributes")))
                return bail(rc);
            if ((rc = ck(stream_configure(R, ctx->smem_optin), "streaming kernel attributes")))
                return bail(rc);
        }
        if ((rc = ck(cudaMalloc(&ctx->dev_err, sizeof(int)), "error word")) ||
            (rc = ck(cudaMemset(ctx->dev_err, 0, sizeof(int)), "error word")) ||
            (rc = ck(cudaMalloc(&ctx->nonfinite, 2 * sizeof(unsigned long long)), "counters")) ||
            (rc = ck(cudaMemset(ctx->nonfinite, 0, 2 * sizeof(unsigned long long)), "counters")))
            return bail(rc);
    }

    if (pso) {
        const empso_pso &p = *pso;
        if (p.P < 1 || p.P > MAX_PSO_P || p.D < 1 || p.D > MAX_PSO_D) {
            ctx->err = "swarm: need 1 <= P <= 2048 and 1 <= D <= 1024";
            return bail(EMPSO_UNSUPPORTED);
        }
        if (!(p.c1 + p.c2 >= 4.0) || !(p.lambda > 0) || !(p.p_em >= 0 && p.p_em <= 1) ||
            !(p.nm_frac >= 0 && p.nm_frac <= 1) || !xmin || !xmax) {
            ctx->err = "swarm: need c1 + c2 >= 4 (Eq. 3), lambda > 0, p_em and nm_frac in [0,1], "
                       "xmin/xmax";
            return bail(EMPSO_INVALID_ARG);
        }
        for (int d = 0; d < p.D; ++d)
            if (!(xmax[d] > xmin[d])) {
                ctx->err = "swarm: need xmax > xmin in every dimension";
                return bail(EMPSO_INVALID_ARG);
            }
        ctx->has_pso = true;
        ctx->pcfg = p;
        const size_t PD = (size_t)p.P * p.D;
        if ((rc = ck(cudaMalloc(&ctx->pso_mem, sizeof(double) * (3 * PD + p.P + 2 * p.D)), "swarm")) ||
            (rc = ck(cudaMalloc(&ctx->pso_int, sizeof(int) * (2 * p.P + 2)), "swarm ints")) ||
            (rc = ck(cudaMalloc(&ctx->xf, sizeof(float) * PD), "positions")) ||
            (rc = ck(cudaMalloc(&ctx->gen_misfit, sizeof(double) * p.P), "generation misfit")))
            return bail(rc);
        PsoDev &s = ctx->pso;
        s.P = p.P;
        s.D = p.D;
        s.NM = (int)std::floor(p.nm_frac * p.P);
        s.em_start = p.em_start;
        s.em_enabled = p.em_enabled;
        s.c1 = p.c1;
        s.c2 = p.c2;
        s.lambda = p.lambda;
        s.p_em = p.p_em;
        s.seed = p.seed;
        s.x = ctx->pso_mem;
        s.v = s.x + PD;
        s.p = s.v + PD;
        s.pf = s.p + PD;
        double *bounds = s.pf + p.P;
        s.xmin = bounds;
        s.xmax = bounds + p.D;
        s.order = ctx->pso_int;
        s.gk = ctx->pso_int + p.P;
        s.rank_of = ctx->pso_int + p.P + 2;
        s.xf = ctx->xf;
        if ((rc = ck(cudaMemcpy(bounds, xmin, sizeof(double) * p.D, cudaMemcpyHostToDevice), "xmin")) ||
            (rc = ck(cudaMemcpy(bounds + p.D, xmax, sizeof(double) * p.D, cudaMemcpyHostToDevice),
                     "xmax")) ||
            (rc = ck(cudaMemset(ctx->pso_int, 0, sizeof(int) * (2 * p.P + 2)), "swarm ints")))
            return bail(rc);
    }
    if ((rc = ck(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking), "capture stream")) ||
        (rc = ck(cudaEventCreateWithFlags(&ctx->chain_fork, cudaEventDisableTiming), "chain event")))
        return bail(rc);
    for (int i = 0; i < empso_ctx::MAX_CHAINS - 1; ++i)
        if ((rc = ck(cudaStreamCreateWithFlags(&ctx->chain_stream[i], cudaStreamNonBlocking), "chain stream")) ||
            (rc = ck(cudaEventCreateWithFlags(&ctx->chain_join[i], cudaEventDisableTiming), "chain event")))
            return bail(rc);
    if ((rc = ck(cudaDeviceSynchronize(), "setup kernels"))) return bail(rc);
    *out = ctx;
    return EMPSO_OK;
}

void empso_destroy(empso_ctx *ctx) { free_ctx(ctx); }

empso_status empso_grid_info(const empso_ctx *ctx, int32_t grid_id, float *dt, int32_t *nt)
{
    if (!ctx) return EMPSO_INVALID_ARG;
    if (grid_id < 0 || grid_id >= (int)ctx->grids.size()) return EMPSO_INVALID_ARG;
    if (dt) *dt = ctx->grids[grid_id].dev.dt;
    if (nt) *nt = ctx->grids[grid_id].dev.nt;
    return EMPSO_OK;
}

empso_status empso_time_axis(const empso_grid *grid, float *dt, int32_t *nt)
{
    g_create_error.clear();
    if (!grid) return fail(nullptr, EMPSO_INVALID_ARG, "null grid");
    GridDev g;
    std::string err;
    const empso_status rc = derive_grid(*grid, 0, g, err);
    if (rc != EMPSO_OK) return fail(nullptr, rc, err);
    if (dt) *dt = g.dt;
    if (nt) *nt = g.nt;
    return EMPSO_OK;
}

empso_status empso_set_levels(empso_ctx *ctx, int32_t grid_id, int32_t n_levels,
                              const float *level_z, const int32_t *level_count, const float *node_x)
{
    if (!ctx) return EMPSO_INVALID_ARG;
    ctx->err.clear();
    if (grid_id < 0 || grid_id >= (int)ctx->grids.size()) return fail(ctx, EMPSO_INVALID_ARG, "bad grid id");
    if (n_levels < 1 || n_levels > MAX_PSO_D || !level_z || !level_count || !node_x)
        return fail(ctx, EMPSO_INVALID_ARG, "need 1 <= n_levels <= 1024 and non-NULL tables");
    std::vector<int> off(n_levels + 1, 0);
    for (int l = 0; l < n_levels; ++l) {
        if (level_count[l] < 1) return fail(ctx, EMPSO_INVALID_ARG, "every level needs a node");
        if (!std::isfinite(level_z[l]) || (l > 0 && !(level_z[l] > level_z[l - 1])))
            return fail(ctx, EMPSO_INVALID_ARG, "level depths must be finite and strictly increasing");
        off[l + 1] = off[l] + level_count[l];
        if (off[l + 1] > MAX_PSO_D) return fail(ctx, EMPSO_UNSUPPORTED, "more than 1024 control nodes");
    }
    for (int l = 0; l < n_levels; ++l)
        for (int k = off[l]; k < off[l + 1]; ++k)
            if (!std::isfinite(node_x[k]) || (k > off[l] && !(node_x[k] > node_x[k - 1])))
                return fail(ctx, EMPSO_INVALID_ARG,
                            "node positions must be finite and strictly increasing within a level");
    const int K = off[n_levels];
    GridHost &G = ctx->grids[grid_id];
    const size_t npts = (size_t)G.dev.nx * G.dev.nz;
    CK(ctx, cudaDeviceSynchronize());
    cudaFree(G.level_z);
    cudaFree(G.node_x);
    cudaFree(G.level_off);
    cudaFree(G.lidx);
    cudaFree(G.lw);
    G.level_z = G.node_x = nullptr;
    G.level_off = nullptr;
    G.lidx = nullptr;
    G.lw = nullptr;
    G.dev.mode = G.spec.interp_mode;   // unchanged until the tables are in place
    CK(ctx, cudaMalloc(&G.level_z, sizeof(float) * n_levels));
    CK(ctx, cudaMalloc(&G.node_x, sizeof(float) * K));
    CK(ctx, cudaMalloc(&G.level_off, sizeof(int) * (n_levels + 1)));
    CK(ctx, cudaMalloc(&G.lidx, sizeof(int4) * npts));
    CK(ctx, cudaMalloc(&G.lw, sizeof(float4) * npts));
    CK(ctx, cudaMemcpy(G.level_z, level_z, sizeof(float) * n_levels, cudaMemcpyHostToDevice));
    CK(ctx, cudaMemcpy(G.node_x, node_x, sizeof(float) * K, cudaMemcpyHostToDevice));
    CK(ctx, cudaMemcpy(G.level_off, off.data(), sizeof(int) * (n_levels + 1), cudaMemcpyHostToDevice));
    G.dev.lidx = G.lidx;
    G.dev.lw = G.lw;
    CK(ctx, launch_level_taps(G.dev, n_levels, G.level_z, G.level_off, G.node_x, G.lidx, G.lw, 0));
    G.dev.mode = 2;
    G.dev.K = K;
    G.spec.interp_mode = 2;
    return grid_changed(ctx, grid_id);
}

empso_status empso_lowpass(empso_ctx *ctx, const float *in, int32_t S, int32_t nt_in, int32_t nrec,
                           double dt_in, float *out, int32_t nt_out, double dt_out, double f_cut,
                           double half_width, void *stream)
{
    if (!ctx) return EMPSO_INVALID_ARG;
    ctx->err.clear();
    if (S < 1 || nt_in < 1 || nrec < 1 || nt_out < 1 || !in || !out || in == out ||
        !(dt_in > 0) || !(dt_out > 0) || !(f_cut > 0) || !(half_width > 0) ||
        !std::isfinite(dt_in) || !std::isfinite(dt_out) || !std::isfinite(f_cut) ||
        !std::isfinite(half_width))
        return fail(ctx, EMPSO_INVALID_ARG,
                    "need positive sizes, finite dt_in, dt_out, f_cut, half_width > 0, in != out");
    if (((double)nt_out * dt_out + half_width) / dt_in > 1e9)
        return fail(ctx, EMPSO_INVALID_ARG, "output times beyond 1e9 input samples");
    const long long span = lowpass_span(dt_in, dt_out, half_width);
    const size_t smem = lowpass_smem_bytes(span);
    if (smem > ctx->smem_optin)
        return fail(ctx, EMPSO_UNSUPPORTED, "filter window too long for shared memory "
                                            "(half_width / dt_in too large)");
    CK(ctx, lowpass_configure(smem));
    CK(ctx, launch_lowpass(in, S, nt_in, nrec, dt_in, out, nt_out, dt_out, f_cut, half_width, smem,
                           (cudaStream_t)stream));
    return EMPSO_OK;
}

}  // extern "C"

namespace {

// grow a device array to at least `need` elements (contents not kept)
template <class T> empso_status adj_grow(empso_ctx *ctx, T **p, size_t *cap, size_t need, bool *grew)
{
    if (*cap >= need) return EMPSO_OK;
    cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    if (cudaMalloc(p, sizeof(T) * std::max<size_t>(need, 1)) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(ctx, EMPSO_OOM, "gradient workspace: " + std::to_string(sizeof(T) * need) + " bytes");
    }
    *cap = need;
    if (grew) *grew = true;
    return EMPSO_OK;
}

// misfit and dphi/dv of M gridded models (all shots on one grid)
// The adjoint-state gradient of M models (and their misfits); with
// forward_only just the misfits, from the gradient's forward pass (the local
// FWI's line search on grids the cluster kernels do not hold).
empso_status gradient_impl(empso_ctx *ctx, const float *vel, int M, const empso_shot *shots, int S,
                           const float *d_obs, double *misfit, float *grad, cudaStream_t st,
                           bool forward_only = false)
{
    const int gid = shots[0].grid_id;
    for (int s = 1; s < S; ++s)
        if (shots[s].grid_id != gid) return fail(ctx, EMPSO_INVALID_ARG, "gradient: all shots on one grid");
    const GridDev &g = ctx->grids[gid].dev;
    const long long I = (long long)M * S;
    const size_t F = (size_t)g.field;
    int rec_max = 0;
    for (int s = 0; s < S; ++s) rec_max = std::max(rec_max, (int)shots[s].nrec);
    auto &W = ctx->adj;
    bool grewH = false;
    empso_status rc;
    if ((rc = adj_grow(ctx, &W.a, &W.a_cap, 2 * F * M, nullptr))) return rc;
    W.B = W.a + F * M;
    if ((rc = adj_grow(ctx, &W.H, &W.H_cap, F * (size_t)(g.nt + 1) * I, &grewH))) return rc;
    // per instance: mu [3], G, J [2]
    // per instance: four adjoint-field slots (the two-step backward rotates
    // through all four, the one-step backward and the per-step forward use
    // two), the gradient, four receiver-term slots
    if ((rc = adj_grow(ctx, &W.mu, &W.mu_cap, F * 9 * I, nullptr))) return rc;
    W.G = W.mu + F * 4 * I;
    // residuals in the modelling trace layout [model][shot][nt][nrec]
    std::vector<long long> doff(S + 1, 0);
    for (int s = 0; s < S; ++s) doff[s + 1] = doff[s] + (long long)g.nt * shots[s].nrec;
    if ((rc = adj_grow(ctx, &W.E, &W.E_cap, (size_t)doff[S] * M, nullptr))) return rc;
    if ((rc = adj_grow(ctx, &W.insts, &W.inst_cap, (size_t)I, nullptr))) return rc;
    if ((rc = adj_grow(ctx, &W.phi, &W.phi_cap, (size_t)I, nullptr))) return rc;
    // zero halo rows and u^0 of the history whenever its layout changes
    std::ostringstream lay;
    lay << gid << "|" << I << "|" << (const void *)W.H;
    if (grewH || W.layout != lay.str()) {
        CK(ctx, cudaMemsetAsync(W.H, 0, sizeof(float) * F * (size_t)(g.nt + 1) * I, st));
        W.layout = lay.str();
    }
    CK(ctx, cudaMemsetAsync(W.mu, 0, sizeof(float) * F * 9 * I, st));
    // The forward pass runs on the on-chip cluster kernel, which streams the
    // history out beside its usual work, when the kernel selection allows it
    // and the grid fits a cluster's shared memory; else one tiled launch per
    // step.  Its cluster size: a gradient has few instances (shots x models),
    // so the rounds of clusters matter, not only the SMs busy: the fewest
    // rounds x rows per CTA (a round's time follows the rows a CTA sweeps),
    // then the most SMs busy, over C <= 12 when some such size fits (13..16
    // measured slower at every shot count: 16 shots on the 461 x 151 grid
    // took 28.5 ms at C = 12, 30.2 at the 15 clusters of C = 9, 31.3-32.4 at
    // C = 13..16).
    int rC = 0, r_threads = 0, r_nc = 0, r_rows = 0;
    size_t r_smem = 0;
    // (the cluster kernels hold stencils up to radius 4: order 16 takes the
    // per-step launches)
    const bool want_res = g.R <= MAX_R_FAST &&
                          (ctx->kernel_kind == EMPSO_KERNEL_AUTO || ctx->kernel_kind == EMPSO_KERNEL_RESIDENT);
    if (want_res) {
        long long best_cost = 0, best_sms = 0;
        // C <= 12 first; 13 .. 16 only for grids that need them
        for (int pass = 0; pass < 2 && !rC; ++pass)
        for (int C = pass == 0 ? 1 : 13; C <= (pass == 0 ? 12 : 16); ++C)
            for (const int rows : resident_runs(ctx->forced_rows)) {
                if (ctx->forced_C > 0 && C != ctx->forced_C) continue;
                if (!resident_fits(g, C, rec_max, ctx->smem_optin, rows)) continue;
                const size_t sm = resident_smem_bytes(g, C, rec_max);
                const int threads = resident_threads(g, C, rows);
                const int nc = (int)std::min<long long>(memo_resident_clusters(g.R, C, threads, sm, rows, true), I);
                if (nc <= 0) continue;
                const long long cost = (I + nc - 1) / nc * (long long)((g.NZ + C - 1) / C);
                const long long sms = (long long)nc * C;
                if (!rC || cost < best_cost || (cost == best_cost && sms > best_sms)) {
                    best_cost = cost;
                    best_sms = sms;
                    rC = C;
                    r_rows = rows;
                    r_threads = threads;
                    r_nc = nc;
                    r_smem = sm;
                }
            }
    }
    if (ctx->kernel_kind == EMPSO_KERNEL_RESIDENT && !rC)
        return fail(ctx, EMPSO_UNSUPPORTED, "gradient: the grid does not fit the on-chip kernel");
    // else the L2 cluster kernel, also streaming the history out, when the
    // selection allows it and the grid fits: the cluster size that keeps the
    // most SMs busy with the instances in flight inside the L2 budget
    int lC = 0, l_threads = 0, l_nc = 0;
    long long l_slot = 0;
    size_t l_smem = 0;
    if (!rC && g.R <= MAX_R_FAST &&
        (ctx->kernel_kind == EMPSO_KERNEL_AUTO || ctx->kernel_kind == EMPSO_KERNEL_CLUSTER_L2)) {
        const size_t sm = l2_smem_bytes(rec_max);
        long long best = 0;
        for (int C : {16, 12, 10, 8, 6, 4, 3, 2, 1}) {
            if (sm > ctx->smem_optin || !l2_fits(g, C)) continue;
            const long long slot = l2_slot_f4(g, C);
            const long long inst_bytes = 32 * slot + 4 * g.field;
            const int rows_c = (g.NZ + C - 1) / C;
            const long long items = std::max<long long>(32, (long long)g.NQ * ((rows_c + 7) / 8));
            const int threads = (int)std::min<long long>(l2_max_threads(), (items + 31) / 32 * 32);
            CK(ctx, l2_configure(g.R, sm, C));
            const int occ = memo_l2_clusters(g.R, C, threads, sm, true);
            if (occ <= 0) continue;
            const long long by_l2 = std::max<long long>(1, L2_BUDGET_BYTES / inst_bytes);
            const int nc = (int)std::min<long long>(std::min<long long>(occ, I), by_l2);
            if ((long long)nc * C > best) {
                best = (long long)nc * C;
                lC = C;
                l_threads = threads;
                l_nc = nc;
                l_slot = slot;
                l_smem = sm;
            }
        }
    }
    if (ctx->kernel_kind == EMPSO_KERNEL_CLUSTER_L2 && !lC)
        return fail(ctx, EMPSO_UNSUPPORTED, "gradient: the grid does not fit the L2 cluster kernel");
    const size_t r_ofs = ((size_t)I * sizeof(Inst) + 255) / 256 * 256;
    const bool table = rC || lC;
    if (table) {
        if ((rc = adj_grow(ctx, &W.rtab, &W.rtab_cap, r_ofs + sizeof(int4) * (size_t)I, nullptr))) return rc;
        if ((rc = adj_grow(ctx, &W.counter, &W.counter_cap, 1, nullptr))) return rc;
    }
    if (lC && (rc = adj_grow(ctx, &W.slots, &W.slots_cap, 2 * (size_t)l_slot * l_nc, nullptr))) return rc;
    // instance tables (the previous call's kernels may still read the old ones)
    std::vector<AdjInst> hi((size_t)I);
    std::vector<unsigned char> rh(table ? r_ofs + sizeof(int4) * (size_t)I : 0);
    for (int m = 0; m < M; ++m)
        for (int s = 0; s < S; ++s) {
            const long long q = (long long)m * S + s;
            AdjInst &in = hi[(size_t)q];
            in.a = W.a + F * m;
            in.B = W.B + F * m;
            in.H = W.H + F * (size_t)(g.nt + 1) * q;
            in.mu = W.mu + F * 4 * q;
            in.G = W.G + F * q;
            in.J = W.mu + F * 5 * I + F * 4 * q;
            in.E = W.E + (size_t)doff[S] * m + doff[s];
            in.dobs = d_obs + doff[s];
            in.rec = ctx->rec_dev + shots[s].rec_begin;
            in.nrec = shots[s].nrec;
            in.sx = shots[s].sx;
            in.sz = shots[s].sz;
            in.w = shots[s].weight;
            // padded rows of the receivers' bilinear corners, one row of margin
            // either side of the device's rounding
            in.jr0 = g.NZ;
            in.jr1 = -1;
            for (int r = 0; r < shots[s].nrec; ++r) {
                const float fz = ctx->rec_host[2 * ((size_t)shots[s].rec_begin + r) + 1] / g.hz + (float)g.pad;
                const int j0 = std::min(std::max((int)std::floor(fz), 0), g.NZ - 2);
                in.jr0 = std::min(in.jr0, j0 - 1);
                in.jr1 = std::max(in.jr1, j0 + 2);
            }
            if (table) {
                Inst ri{};
                ri.a = in.a;
                ri.dobs = nullptr;        // traces only; the residual kernel subtracts d_obs
                ri.traces = in.E;
                ri.rec = in.rec;
                ri.grid = gid;
                ri.nrec = in.nrec;
                ri.sx = in.sx;
                ri.sz = in.sz;
                ri.out = (int)q;
                ri.hist = in.H;
                reinterpret_cast<Inst *>(rh.data())[q] = ri;
                reinterpret_cast<int4 *>(rh.data() + r_ofs)[q] = make_int4((int)q, -1, 0, 0);
            }
        }
    CK(ctx, cudaStreamSynchronize(st));
    CK(ctx, cudaMemcpy(W.insts, hi.data(), sizeof(AdjInst) * hi.size(), cudaMemcpyHostToDevice));
    if (table) CK(ctx, cudaMemcpy(W.rtab, rh.data(), rh.size(), cudaMemcpyHostToDevice));
    const int rec_threads = std::min(1024, std::max(32, (rec_max + 31) / 32 * 32));
    CK(ctx, launch_vel_to_field(g, vel, M, W.a, g.field, st));
    CK(ctx, launch_adj_prep(g, W.a, W.B, M, st));
    // the two time loops replay as one graph
    std::ostringstream key;
    key << gid << "|" << I << "|" << rec_threads << "|" << (const void *)W.insts << "|" << rC << "|" << lC
        << "|" << (const void *)W.rtab << "|" << (const void *)W.slots << "|" << forward_only << "|"
        << ctx->grad_chains;
    cudaGraphExec_t exec = nullptr;
    for (auto &e : W.graphs)
        if (e.first == key.str()) exec = e.second;
    if (!exec) {
        cudaGraph_t graph = nullptr;
        CK(ctx, cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
        cudaError_t ce;
        if (rC) {
            ce = cudaMemsetAsync(W.counter, 0, sizeof(int), ctx->cap_stream);
            if (ce == cudaSuccess)
                ce = launch_wave_resident(g.R, ctx->grids_dev, reinterpret_cast<const Inst *>(W.rtab),
                                          reinterpret_cast<const int4 *>(W.rtab + r_ofs), (int)I, false,
                                          W.counter, rC, r_nc, r_threads, r_rows, rec_max, r_smem, W.phi,
                                          ctx->cap_stream, true);
            if (ce == cudaSuccess) ce = launch_adj_residual(g, W.insts, (int)I, rec_max, ctx->cap_stream);
        } else if (lC) {
            ce = cudaMemsetAsync(W.counter, 0, sizeof(int), ctx->cap_stream);
            if (ce == cudaSuccess)
                ce = launch_wave_l2(g.R, ctx->grids_dev, reinterpret_cast<const Inst *>(W.rtab), (int)I, W.counter,
                                    lC, l_nc, l_threads, W.slots, l_slot, rec_max, l_smem, W.phi,
                                    ctx->cap_stream, true);
            if (ce == cudaSuccess) ce = launch_adj_residual(g, W.insts, (int)I, rec_max, ctx->cap_stream);
        } else {
            // the per-step forward pass with its time levels in the (zeroed)
            // adjoint slots and L u^n as the history; the slots are zeroed
            // again for the backward pass
            ce = launch_adj_forward(g, W.insts, (int)I, rec_threads, ctx->cap_stream);
            if (ce == cudaSuccess && !forward_only)
                ce = cudaMemsetAsync(W.mu, 0, sizeof(float) * F * 4 * I, ctx->cap_stream);
        }
        if (ce == cudaSuccess && !forward_only) {
            // instances [c I / n, (c + 1) I / n) on chain c (chain 0 on the
            // capture stream), forked after the forward pass and joined at the end
            const int want = ctx->grad_chains > 0 ? ctx->grad_chains : (I >= 16 ? 4 : 1);
            const int n = (int)std::max<long long>(1, std::min<long long>(want, I));
            if (n > 1) ce = cudaEventRecord(ctx->chain_fork, ctx->cap_stream);
            for (int c = 1; c < n && ce == cudaSuccess; ++c)
                ce = cudaStreamWaitEvent(ctx->chain_stream[c - 1], ctx->chain_fork, 0);
            for (int c = 0; c < n && ce == cudaSuccess; ++c) {
                const long long i0 = c * I / n, i1 = (c + 1) * I / n;
                ce = launch_adj_backward(g, W.insts + i0, (int)(i1 - i0), (int)I, rec_threads,
                                         c == 0 ? ctx->cap_stream : ctx->chain_stream[c - 1]);
            }
            for (int c = 1; c < n && ce == cudaSuccess; ++c) {
                ce = cudaEventRecord(ctx->chain_join[c - 1], ctx->chain_stream[c - 1]);
                if (ce == cudaSuccess) ce = cudaStreamWaitEvent(ctx->cap_stream, ctx->chain_join[c - 1], 0);
            }
        }
        const cudaError_t ee = cudaStreamEndCapture(ctx->cap_stream, &graph);
        if (ce == cudaSuccess) ce = ee;
        if (ce == cudaSuccess) ce = cudaGraphInstantiate(&exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (ce != cudaSuccess)
            return fail(ctx, EMPSO_CUDA_ERROR, std::string("gradient graph: ") + cudaGetErrorString(ce));
        W.graphs.push_back({key.str(), exec});
    }
    CK(ctx, cudaGraphLaunch(exec, st));
    if (forward_only) {
        CK(ctx, launch_adj_misfit(g, W.insts, M, S, W.phi, misfit, reinterpret_cast<double *>(W.mu), st));
        return EMPSO_OK;
    }
    // the fold's scratch takes the adjoint fields' slots (free now; G lies past them)
    CK(ctx, launch_adj_finish(g, W.insts, M, S, vel, W.phi, misfit, grad, W.mu, st));
    return EMPSO_OK;
}

}  // namespace

extern "C" {

empso_status empso_gradient(empso_ctx *ctx, const float *vel, int32_t M, const empso_shot *shots,
                            int32_t S, const float *d_obs, double *misfit, float *grad, void *stream)
{
    if (!ctx) return EMPSO_INVALID_ARG;
    ctx->err.clear();
    if (M < 1 || !vel || !d_obs || !grad) return fail(ctx, EMPSO_INVALID_ARG, "bad vel/d_obs/grad");
    empso_status rc = check_shots(ctx, shots, S, shots && S > 0 ? shots[0].grid_id : -1);
    if (rc) return rc;
    return gradient_impl(ctx, vel, M, shots, S, d_obs, misfit, grad, (cudaStream_t)stream);
}

empso_status empso_fwi(empso_ctx *ctx, float *vel, const empso_shot *shots, int32_t S,
                       const float *d_obs, int32_t iters, float vmin, float vmax, double *history,
                       int32_t *done, void *stream)
{
    if (!ctx) return EMPSO_INVALID_ARG;
    ctx->err.clear();
    if (!vel || !d_obs || iters < 0 || !(vmin > 0) || !(vmin <= vmax))
        return fail(ctx, EMPSO_INVALID_ARG, "bad vel/d_obs/iters/bounds");
    empso_status rc = check_shots(ctx, shots, S, shots && S > 0 ? shots[0].grid_id : -1);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const GridDev &g = ctx->grids[shots[0].grid_id].dev;
    const int np = g.nx * g.nz;
    auto &W = ctx->adj;
    if ((rc = adj_grow(ctx, &W.fv, &W.fv_cap, (size_t)3 * np, nullptr))) return rc;
    if (!W.fd) CK(ctx, cudaMalloc(&W.fd, sizeof(double) * 16));
    float *vt = W.fv, *gcur = W.fv + np, *gnew = W.fv + 2 * (size_t)np;
    double *dots = W.fd, *phi_dev = W.fd + 8;
    double r[5];
    // misfits on the modelling kernels, or, for stencils the cluster kernels do
    // not hold (order 16), on the gradient's tiled forward pass over every SM
    const bool fwd_misfit = g.R > MAX_R_FAST;
    auto misfit_of = [&](const float *v, double *out) -> empso_status {
        Models mod;
        mod.vel = v;
        mod.M = 1;
        empso_status e = fwd_misfit ? gradient_impl(ctx, v, 1, shots, S, d_obs, phi_dev, nullptr, st, true)
                                    : run_batch(ctx, mod, shots, S, d_obs, nullptr, phi_dev, st);
        if (e) return e;
        CK(ctx, cudaMemcpyAsync(out, phi_dev, sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(ctx, cudaStreamSynchronize(st));
        return EMPSO_OK;
    };
    auto reduce = [&](const float *a, const float *b, const float *c, const float *d) -> empso_status {
        CK(ctx, launch_fwi_dots(a, b, c, d, np, dots, st));
        CK(ctx, cudaMemcpyAsync(r, dots, sizeof r, cudaMemcpyDeviceToHost, st));
        CK(ctx, cudaStreamSynchronize(st));
        return EMPSO_OK;
    };
    double phi;
    if ((rc = misfit_of(vel, &phi))) return rc;
    if (history) history[0] = phi;
    if ((rc = gradient_impl(ctx, vel, 1, shots, S, d_obs, nullptr, gcur, st))) return rc;
    // first step: the largest model change is 1 % of the mean velocity
    if ((rc = reduce(vel, nullptr, gcur, nullptr))) return rc;
    double alpha = r[3] > 0 ? 0.01 * (r[4] / np) / r[3] : 0.0;
    int it = 0;
    for (; it < iters && alpha > 0; ++it) {
        bool ok = false;
        double phi_t = phi;
        for (int tries = 0; tries < 10 && !ok; ++tries) {
            CK(ctx, launch_fwi_step(vel, gcur, (float)alpha, vmin, vmax, vt, np, st));
            if ((rc = misfit_of(vt, &phi_t))) return rc;
            // Armijo on the step actually taken (after the clip): g . (v - v_t)
            if ((rc = reduce(vel, vt, gcur, nullptr))) return rc;
            const double decrease = r[0];
            if (decrease > 0 && std::isfinite(phi_t) && phi_t <= phi - 1e-4 * decrease) ok = true;
            else alpha *= 0.5;
        }
        if (!ok) break;
        if ((rc = gradient_impl(ctx, vt, 1, shots, S, d_obs, nullptr, gnew, st))) return rc;
        // Barzilai-Borwein step: s = v_t - v, y = g_new - g; alpha = s.s / s.y
        if ((rc = reduce(vt, vel, gnew, gcur))) return rc;
        const double ss = r[1], sy = r[2];
        if (sy > 0) alpha = ss / sy;
        CK(ctx, cudaMemcpyAsync(vel, vt, sizeof(float) * np, cudaMemcpyDeviceToDevice, st));
        CK(ctx, cudaMemcpyAsync(gcur, gnew, sizeof(float) * np, cudaMemcpyDeviceToDevice, st));
        phi = phi_t;
        if (history) history[it + 1] = phi;
    }
    CK(ctx, cudaStreamSynchronize(st));
    if (done) *done = it;
    return EMPSO_OK;
}

empso_status empso_set_water(empso_ctx *ctx, int32_t grid_id, float water_depth, float v_water)
{
    if (!ctx) return EMPSO_INVALID_ARG;
    ctx->err.clear();
    if (grid_id < 0 || grid_id >= (int)ctx->grids.size()) return fail(ctx, EMPSO_INVALID_ARG, "bad grid id");
    if (!std::isfinite(water_depth) || !(v_water > 0) || !std::isfinite(v_water))
        return fail(ctx, EMPSO_INVALID_ARG, "need a finite depth and a positive velocity");
    GridHost &G = ctx->grids[grid_id];
    G.dev.water_z = water_depth > 0.f ? water_depth : 0.f;
    G.dev.v_water = v_water;
    return grid_changed(ctx, grid_id);
}

empso_status empso_level_bounds(int32_t n_levels, const float *level_z, const int32_t *level_count,
                                double v_first, double v_last, double lo_first, double hi_first,
                                double lo_last, double hi_last, double *xmin, double *xmax)
{
    if (n_levels < 1 || !level_z || !level_count || !xmin || !xmax) return EMPSO_INVALID_ARG;
    for (int l = 0; l < n_levels; ++l)
        if (level_count[l] < 1 || (l > 0 && !(level_z[l] > level_z[l - 1]))) return EMPSO_INVALID_ARG;
    const double min0 = v_first * (1.0 - lo_first), max0 = v_first * (1.0 + hi_first);
    const double min1 = v_last * (1.0 - lo_last), max1 = v_last * (1.0 + hi_last);
    if (!(min0 <= max0) || !(min1 <= max1)) return EMPSO_INVALID_ARG;
    const double span = (double)level_z[n_levels - 1] - (double)level_z[0];
    long long k = 0;
    for (int l = 0; l < n_levels; ++l) {
        // position of the level between the first (0) and the last (1) in depth
        const double s = n_levels > 1 ? ((double)level_z[l] - (double)level_z[0]) / span : 0.0;
        const double lo = min0 + s * (min1 - min0), hi = max0 + s * (max1 - max0);
        for (int i = 0; i < level_count[l]; ++i, ++k) {
            xmin[k] = lo;
            xmax[k] = hi;
        }
    }
    return EMPSO_OK;
}

empso_status empso_interp(empso_ctx *ctx, int32_t grid_id, const float *particles, int32_t P,
                          float *vel_out, void *stream)
{
    if (!ctx) return EMPSO_INVALID_ARG;
    ctx->err.clear();
    if (grid_id < 0 || grid_id >= (int)ctx->grids.size())
        return fail(ctx, EMPSO_INVALID_ARG, "grid_id out of range");
    if (P < 0 || (P > 0 && (!particles || !vel_out)))
        return fail(ctx, EMPSO_INVALID_ARG, "bad particles/vel_out");
    if (P == 0) return EMPSO_OK;
    const GridDev &g = ctx->grids[grid_id].dev;
    empso_status rc = grow(ctx, (void **)&ctx->fields, &ctx->fields_cap,
                           sizeof(float) * g.field * P, sizeof(float));
    if (rc) return rc;
    CK(ctx, launch_interp(g, particles, P, ctx->fields, g.field, vel_out, (cudaStream_t)stream));
    return EMPSO_OK;
}

empso_status forward_traces(empso_ctx *ctx, const float *vel, int32_t M, const empso_shot *shots,
                            int32_t S, float *traces, void *stream)
{
    if (!ctx) return EMPSO_INVALID_ARG;
    ctx->err.clear();
    if (M < 0 || (M > 0 && (!vel || !traces))) return fail(ctx, EMPSO_INVALID_ARG, "bad vel/traces");
    empso_status rc = check_shots(ctx, shots, S, shots && S > 0 ? shots[0].grid_id : -1);
    if (rc || M == 0) return rc;
    Models mod;
    mod.vel = vel;
    mod.M = M;
    return run_batch(ctx, mod, shots, S, nullptr, traces, nullptr, (cudaStream_t)stream);
}

empso_status eval_models(empso_ctx *ctx, const float *vel, int32_t M, const empso_shot *shots,
                         int32_t S, const float *d_obs, double *misfit, void *stream)
{
    if (!ctx) return EMPSO_INVALID_ARG;
    ctx->err.clear();
    if (M < 0 || (M > 0 && (!vel || !d_obs || !misfit)))
        return fail(ctx, EMPSO_INVALID_ARG, "bad vel/d_obs/misfit");
    empso_status rc = check_shots(ctx, shots, S, shots && S > 0 ? shots[0].grid_id : -1);
    if (rc || M == 0) return rc;
    Models mod;
    mod.vel = vel;
    mod.M = M;
    cudaStream_t st = (cudaStream_t)stream;
    if ((rc = strict_begin(ctx, st))) return rc;
    return strict_end(ctx, run_batch(ctx, mod, shots, S, d_obs, nullptr, misfit, st), st);
}

empso_status eval_fitness(empso_ctx *ctx, const float *particles, int32_t P,
                          const empso_shot *shots, int32_t S, const float *d_obs, double *misfit,
                          void *stream)
{
    if (!ctx) return EMPSO_INVALID_ARG;
    ctx->err.clear();
    if (P < 0 || (P > 0 && (!particles || !d_obs || !misfit)))
        return fail(ctx, EMPSO_INVALID_ARG, "bad particles/d_obs/misfit");
    empso_status rc = check_shots(ctx, shots, S, -1);
    if (rc || P == 0) return rc;
    const int K = ctx->grids[shots[0].grid_id].dev.K;
    for (int s = 1; s < S; ++s) {
        if (ctx->grids[shots[s].grid_id].dev.K != K)
            return fail(ctx, EMPSO_INVALID_ARG, "shots' grids disagree on the control nodes");
    }
    Models mod;
    mod.particles = particles;
    mod.M = P;
    cudaStream_t st = (cudaStream_t)stream;
    if ((rc = strict_begin(ctx, st))) return rc;
    return strict_end(ctx, run_batch(ctx, mod, shots, S, d_obs, nullptr, misfit, st), st);
}

empso_status pso_init(empso_ctx *ctx, float *particles_out, void *stream)
{
    if (!ctx) return EMPSO_INVALID_ARG;
    ctx->err.clear();
    if (!ctx->has_pso) return fail(ctx, EMPSO_NOT_INITIALIZED, "context has no swarm");
    CK(ctx, launch_pso_init(ctx->pso, particles_out, (cudaStream_t)stream));
    return EMPSO_OK;
}

empso_status pso_step(empso_ctx *ctx, const double *misfit, float *particles_out,
                      int32_t *gbest_out, void *stream)
{
    if (!ctx) return EMPSO_INVALID_ARG;
    ctx->err.clear();
    if (!ctx->has_pso) return fail(ctx, EMPSO_NOT_INITIALIZED, "context has no swarm");
    if (!misfit) return fail(ctx, EMPSO_INVALID_ARG, "misfit is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    CK(ctx, launch_pso_step(ctx->pso, misfit, particles_out, st));
    if (gbest_out) {
        CK(ctx, cudaMemcpyAsync(gbest_out, ctx->pso.gk, sizeof(int), cudaMemcpyDeviceToHost, st));
        CK(ctx, cudaStreamSynchronize(st));
    }
    return EMPSO_OK;
}

empso_status pso_get_state(empso_ctx *ctx, double *x, double *v, double *p, double *pf,
                           int32_t *order, int32_t *gk, void *stream)
{
    if (!ctx) return EMPSO_INVALID_ARG;
    ctx->err.clear();
    if (!ctx->has_pso) return fail(ctx, EMPSO_NOT_INITIALIZED, "context has no swarm");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t PD = sizeof(double) * ctx->pso.P * ctx->pso.D;
    if (x) CK(ctx, cudaMemcpyAsync(x, ctx->pso.x, PD, cudaMemcpyDeviceToDevice, st));
    if (v) CK(ctx, cudaMemcpyAsync(v, ctx->pso.v, PD, cudaMemcpyDeviceToDevice, st));
    if (p) CK(ctx, cudaMemcpyAsync(p, ctx->pso.p, PD, cudaMemcpyDeviceToDevice, st));
    if (pf)
        CK(ctx, cudaMemcpyAsync(pf, ctx->pso.pf, sizeof(double) * ctx->pso.P,
                                cudaMemcpyDeviceToDevice, st));
    if (order)
        CK(ctx, cudaMemcpyAsync(order, ctx->pso.order, sizeof(int) * ctx->pso.P,
                                cudaMemcpyDeviceToDevice, st));
    if (gk) CK(ctx, cudaMemcpyAsync(gk, ctx->pso.gk, 2 * sizeof(int), cudaMemcpyDeviceToDevice, st));
    return EMPSO_OK;
}

empso_status pso_set_state(empso_ctx *ctx, const double *x, const double *v, const double *p,
                           const double *pf, int32_t g, int32_t k, void *stream)
{
    if (!ctx) return EMPSO_INVALID_ARG;
    ctx->err.clear();
    if (!ctx->has_pso) return fail(ctx, EMPSO_NOT_INITIALIZED, "context has no swarm");
    if (!x || !v || !p || !pf) return fail(ctx, EMPSO_INVALID_ARG, "state buffers are NULL");
    if (g < 0 || g >= ctx->pso.P || k < 0) return fail(ctx, EMPSO_INVALID_ARG, "bad g or k");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t PD = sizeof(double) * ctx->pso.P * ctx->pso.D;
    CK(ctx, cudaMemcpyAsync(ctx->pso.x, x, PD, cudaMemcpyDeviceToDevice, st));
    CK(ctx, cudaMemcpyAsync(ctx->pso.v, v, PD, cudaMemcpyDeviceToDevice, st));
    CK(ctx, cudaMemcpyAsync(ctx->pso.p, p, PD, cudaMemcpyDeviceToDevice, st));
    CK(ctx, cudaMemcpyAsync(ctx->pso.pf, pf, sizeof(double) * ctx->pso.P, cudaMemcpyDeviceToDevice,
                            st));
    int gk[2] = {g, k};
    // staged through pinned memory so the copy is stream-ordered
    CK(ctx, cudaEventSynchronize(ctx->stage_free));
    empso_status rc = grow_stage(ctx, 64);
    if (rc) return rc;
    memcpy(ctx->stage_host, gk, sizeof gk);
    CK(ctx, cudaMemcpyAsync(ctx->pso.gk, ctx->stage_host, sizeof gk, cudaMemcpyHostToDevice, st));
    CK(ctx, cudaEventRecord(ctx->stage_free, st));
    CK(ctx, launch_xf_from_x(ctx->pso, st));
    return EMPSO_OK;
}

empso_status empso_generation(empso_ctx *ctx, const empso_shot *shots, int32_t S,
                              const float *d_obs, double *misfit_out, void *stream)
{
    if (!ctx) return EMPSO_INVALID_ARG;
    ctx->err.clear();
    if (!ctx->has_pso) return fail(ctx, EMPSO_NOT_INITIALIZED, "context has no swarm");
    if (!d_obs) return fail(ctx, EMPSO_INVALID_ARG, "d_obs is NULL");
    empso_status rc = check_shots(ctx, shots, S, -1);
    if (rc) return rc;
    for (int s = 0; s < S; ++s) {
        if (ctx->grids[shots[s].grid_id].dev.K != ctx->pso.D)
            return fail(ctx, EMPSO_INVALID_ARG, "swarm dimension differs from the grids' control nodes");
    }
    cudaStream_t st = (cudaStream_t)stream;
    // the captured graph depends on the shots, the buffers, the kernel choice
    // and whether kernel timing is on
    std::string key = batch_key(ctx, shots, S, ctx->pso.P);
    {
        std::ostringstream os;
        os << "|" << (const void *)d_obs << "|" << (const void *)misfit_out << "|k" << ctx->kernel_kind
           << "c" << ctx->forced_C << "r" << ctx->forced_rows << "t" << ctx->timing;
        auto tu = ctx->tuned.find(key);
        if (tu != ctx->tuned.end())
            os << "|tuned" << tu->second.kind << "," << tu->second.C << "," << tu->second.rows;
        for (int s = 0; s < S; ++s)
            os << "|" << shots[s].sx << "," << shots[s].sz << "," << shots[s].rec_begin << ","
               << shots[s].nrec << "," << shots[s].grid_id << "," << shots[s].weight;
        key += os.str();
    }
    empso_ctx::GraphEntry *ge = nullptr;
    for (auto &e : ctx->graphs)
        if (e.key == key) ge = &e;
    if (!ge) {
        Models mod;
        mod.particles = ctx->xf;
        mod.M = ctx->pso.P;
        empso_ctx::GraphEntry e;
        e.key = key;
        CK(ctx, cudaMalloc(&e.table, table_bytes((long long)ctx->pso.P * S, S)));
        Plan p;
        // planning allocates and uploads outside the capture; the graph holds
        // only kernels and a memset
        CK(ctx, cudaStreamSynchronize(st));
        if ((rc = plan_batch(ctx, mod, shots, S, d_obs, nullptr, p, e.table, ctx->cap_stream))) {
            cudaFree(e.table);
            return rc;
        }
        cudaGraph_t graph = nullptr;
        CK(ctx, cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
        rc = enqueue_batch(ctx, mod, p, ctx->gen_misfit, ctx->cap_stream);
        cudaError_t ce = cudaSuccess;
        if (!rc) ce = launch_pso_step(ctx->pso, ctx->gen_misfit, nullptr, ctx->cap_stream);
        if (!rc && ce == cudaSuccess && misfit_out)
            ce = cudaMemcpyAsync(misfit_out, ctx->gen_misfit, sizeof(double) * ctx->pso.P,
                                 cudaMemcpyDeviceToDevice, ctx->cap_stream);
        cudaError_t ee = cudaStreamEndCapture(ctx->cap_stream, &graph);
        if (rc || ce != cudaSuccess || ee != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            cudaFree(e.table);
            if (rc) return rc;
            return fail(ctx, EMPSO_CUDA_ERROR, std::string("graph capture: ") +
                                                  cudaGetErrorString(ce != cudaSuccess ? ce : ee));
        }
        ce = cudaGraphInstantiate(&e.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ce != cudaSuccess) {
            cudaFree(e.table);
            return fail(ctx, EMPSO_CUDA_ERROR, std::string("graph instantiate: ") + cudaGetErrorString(ce));
        }
        ctx->graphs.push_back(e);
        ge = &ctx->graphs.back();
    }
    if ((rc = strict_begin(ctx, st))) return rc;
    CK(ctx, cudaGraphLaunch(ge->exec, st));
    return strict_end(ctx, EMPSO_OK, st);
}

namespace {

// JSON-lines tuning cache: one {"gpu", "key", "kind", "cluster", "ms"} object
// per line; later lines override earlier ones.
std::string gpu_name(int dev)
{
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return "unknown";
    return prop.name;
}

std::string json_str(const std::string &line, const std::string &field)
{
    const std::string pat = "\"" + field + "\": \"";
    size_t a = line.find(pat);
    if (a == std::string::npos) return "";
    a += pat.size();
    size_t b = line.find('"', a);
    return b == std::string::npos ? "" : line.substr(a, b - a);
}

long json_int(const std::string &line, const std::string &field, long dflt)
{
    const std::string pat = "\"" + field + "\": ";
    size_t a = line.find(pat);
    if (a == std::string::npos) return dflt;
    return strtol(line.c_str() + a + pat.size(), nullptr, 10);
}

void load_tune_cache(empso_ctx *ctx)
{
    std::ifstream in(ctx->tune_cache);
    const std::string gpu = gpu_name(ctx->device);
    std::string line;
    while (std::getline(in, line)) {
        if (json_str(line, "gpu") != gpu) continue;
        const std::string key = json_str(line, "key");
        if (key.empty()) continue;
        empso_ctx::Tuned t;
        t.kind = (int)json_int(line, "kind", 0);
        t.C = (int)json_int(line, "cluster", 0);
        t.rows = (int)json_int(line, "rows", 0);
        ctx->tuned[key] = t;
    }
}

}  // namespace

empso_status empso_set_tuning_cache(empso_ctx *ctx, const char *path)
{
    if (!ctx) return EMPSO_INVALID_ARG;
    ctx->err.clear();
    ctx->tune_cache = path ? path : "";
    if (!ctx->tune_cache.empty()) load_tune_cache(ctx);
    return EMPSO_OK;
}

empso_status empso_autotune(empso_ctx *ctx, const float *particles, int32_t P,
                            const empso_shot *shots, int32_t S, const float *d_obs,
                            double *misfit, int32_t *kind_out, int32_t *cluster_out, void *stream)
{
    if (!ctx) return EMPSO_INVALID_ARG;
    ctx->err.clear();
    if (P <= 0 || !particles || !d_obs || !misfit)
        return fail(ctx, EMPSO_INVALID_ARG, "bad particles/d_obs/misfit");
    empso_status rc = check_shots(ctx, shots, S, -1);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const std::string key = batch_key(ctx, shots, S, P);
    ctx->tuned.erase(key);
    const int save_kind = ctx->kernel_kind, save_C = ctx->forced_C, save_rows = ctx->forced_rows;
    Models mod;
    mod.particles = particles;
    mod.M = P;
    cudaEvent_t e0, e1;
    CK(ctx, cudaEventCreate(&e0));
    CK(ctx, cudaEventCreate(&e1));
    // candidates: the streaming kernel, every cluster size and rows-per-thread
    // shape of the on-chip one, and the usual cluster sizes of the L2 one
    // (only those of the selected kind when a kind is selected)
    const int only = ctx->kernel_kind;
    std::vector<empso_ctx::Tuned> cand;
    if (only == EMPSO_KERNEL_AUTO || only == EMPSO_KERNEL_STREAMING) cand.push_back({EMPSO_KERNEL_STREAMING, 0, 0});
    if (only == EMPSO_KERNEL_AUTO || only == EMPSO_KERNEL_RESIDENT)
        for (int C = 1; C <= 16; ++C)
            for (const int rows : RESIDENT_RUNS) cand.push_back({EMPSO_KERNEL_RESIDENT, C, rows});
    if (only == EMPSO_KERNEL_AUTO || only == EMPSO_KERNEL_CLUSTER_L2)
        for (int C : {4, 8, 10, 12, 16}) cand.push_back({EMPSO_KERNEL_CLUSTER_L2, C, 0});
    float best = 1e30f;
    empso_ctx::Tuned choice;
    choice.kind = EMPSO_KERNEL_AUTO;
    for (auto &c : cand) {
        ctx->kernel_kind = c.kind;
        ctx->forced_C = c.C;
        ctx->forced_rows = c.rows;
        Plan p;
        rc = plan_batch(ctx, mod, shots, S, d_obs, nullptr, p, nullptr, st);
        if (rc == EMPSO_UNSUPPORTED) continue;   // this size does not fit the batch
        if (rc) break;
        if ((rc = enqueue_batch(ctx, mod, p, misfit, st))) break;   // warm-up
        cudaEventRecord(e0, st);
        if ((rc = enqueue_batch(ctx, mod, p, misfit, st))) break;
        cudaEventRecord(e1, st);
        cudaError_t ce = cudaEventSynchronize(e1);
        if (ce != cudaSuccess) {
            rc = fail(ctx, EMPSO_CUDA_ERROR, cudaGetErrorString(ce));
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) {
            best = ms;
            choice.kind = c.kind;
            choice.C = p.resident ? p.resC : (p.l2 ? p.l2C : 0);
            choice.rows = p.resident ? p.res_rows : 0;
        }
    }
    ctx->err.clear();
    ctx->kernel_kind = save_kind;
    ctx->forced_C = save_C;
    ctx->forced_rows = save_rows;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc && rc != EMPSO_UNSUPPORTED) return rc;
    if (choice.kind == EMPSO_KERNEL_AUTO) return fail(ctx, EMPSO_UNSUPPORTED, "no kernel fits the batch");
    ctx->tuned[key] = choice;
    if (kind_out) *kind_out = choice.kind;
    if (cluster_out) *cluster_out = choice.C;
    if (!ctx->tune_cache.empty()) {
        std::ofstream out(ctx->tune_cache, std::ios::app);
        out << "{\"gpu\": \"" << gpu_name(ctx->device) << "\", \"key\": \"" << key
            << "\", \"kind\": " << choice.kind << ", \"cluster\": " << choice.C
            << ", \"rows\": " << choice.rows << ", \"ms\": " << best << "}\n";
    }
    return EMPSO_OK;
}

empso_status empso_set_kernel(empso_ctx *ctx, int32_t kind)
{
    if (!ctx) return EMPSO_INVALID_ARG;
    ctx->err.clear();
    if (kind != EMPSO_KERNEL_AUTO && kind != EMPSO_KERNEL_STREAMING && kind != EMPSO_KERNEL_RESIDENT &&
        kind != EMPSO_KERNEL_CLUSTER_L2)
        return fail(ctx, EMPSO_INVALID_ARG, "unknown kernel kind");
    ctx->kernel_kind = kind;
    return EMPSO_OK;
}

empso_status empso_set_cluster(empso_ctx *ctx, int32_t ctas)
{
    if (!ctx) return EMPSO_INVALID_ARG;
    ctx->err.clear();
    if (ctas < 0 || ctas > 16) return fail(ctx, EMPSO_INVALID_ARG, "cluster size must be 0..16");
    ctx->forced_C = ctas;
    return EMPSO_OK;
}

empso_status empso_set_gradient_chains(empso_ctx *ctx, int32_t chains)
{
    if (!ctx) return EMPSO_INVALID_ARG;
    ctx->err.clear();
    if (chains < 0 || chains > empso_ctx::MAX_CHAINS)
        return fail(ctx, EMPSO_INVALID_ARG, "gradient chains must be 0..8");
    ctx->grad_chains = chains;
    return EMPSO_OK;
}

empso_status empso_set_tile_rows(empso_ctx *ctx, int32_t rows)
{
    if (!ctx) return EMPSO_INVALID_ARG;
    ctx->err.clear();
    if (rows != 0 && !resident_rows_supported(rows))
        return fail(ctx, EMPSO_INVALID_ARG, "rows per thread must be 0 (automatic) or 4..13");
    ctx->forced_rows = rows;
    return EMPSO_OK;
}

empso_status empso_last_clusters(const empso_ctx *ctx, int32_t *groups)
{
    if (!ctx || !groups) return EMPSO_INVALID_ARG;
    *groups = ctx->last_groups;
    return EMPSO_OK;
}

empso_status empso_last_tile_rows(const empso_ctx *ctx, int32_t *rows)
{
    if (!ctx || !rows) return EMPSO_INVALID_ARG;
    *rows = ctx->last_path == 2 ? ctx->last_rows : 0;
    return EMPSO_OK;
}

empso_status empso_last_launch(const empso_ctx *ctx, int32_t *kind, int32_t *cluster)
{
    if (!ctx) return EMPSO_INVALID_ARG;
    if (kind)
        *kind = ctx->last_path == 3 ? EMPSO_KERNEL_STREAMING
                                    : (ctx->last_path == 4 ? EMPSO_KERNEL_CLUSTER_L2 : ctx->last_path);
    if (cluster) *cluster = ctx->last_C;
    return EMPSO_OK;
}

empso_status empso_last_paired_units(const empso_ctx *ctx, int32_t *paired)
{
    if (!ctx || !paired) return EMPSO_INVALID_ARG;
    *paired = ctx->last_path == 2 ? ctx->last_paired : 0;
    return EMPSO_OK;
}

const char *empso_last_kernel_name(const empso_ctx *ctx)
{
    if (!ctx) return "";
    switch (ctx->last_path) {
    case 1: return "wave_kernel";
    case 2: return "wave_resident_kernel";
    case 3: return "wave_stream_kernel";
    case 4: return "wave_l2_kernel";
    default: return "";
    }
}

empso_status empso_device_error(empso_ctx *ctx, int32_t *status, void *stream)
{
    if (!ctx || !status) return EMPSO_INVALID_ARG;
    ctx->err.clear();
    cudaStream_t st = (cudaStream_t)stream;
    int v = 0;
    CK(ctx, cudaMemcpyAsync(&v, ctx->dev_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(ctx, cudaStreamSynchronize(st));
    CK(ctx, cudaMemsetAsync(ctx->dev_err, 0, sizeof(int), st));
    *status = v;
    return EMPSO_OK;
}

empso_status empso_set_timing(empso_ctx *ctx, int32_t enable)
{
    if (!ctx) return EMPSO_INVALID_ARG;
    ctx->err.clear();
    if (enable && !ctx->tev[0])
        for (auto &e : ctx->tev) CK(ctx, cudaEventCreate(&e));
    ctx->timing = enable != 0;
    ctx->timed = false;
    return EMPSO_OK;
}

empso_status empso_read_timing(empso_ctx *ctx, double *ms3)
{
    if (!ctx || !ms3) return EMPSO_INVALID_ARG;
    ctx->err.clear();
    if (!ctx->timed) return fail(ctx, EMPSO_NOT_INITIALIZED, "no timed call yet");
    CK(ctx, cudaEventSynchronize(ctx->tev[3]));
    for (int i = 0; i < 3; ++i) {
        float ms = 0.f;
        CK(ctx, cudaEventElapsedTime(&ms, ctx->tev[i], ctx->tev[i + 1]));
        ms3[i] = ms;
    }
    return EMPSO_OK;
}

empso_status pso_step_ranked(empso_ctx *ctx, const double *misfit, const double *rank,
                             float *particles_out, int32_t *gbest_out, void *stream)
{
    if (!ctx) return EMPSO_INVALID_ARG;
    ctx->err.clear();
    if (!ctx->has_pso) return fail(ctx, EMPSO_NOT_INITIALIZED, "context has no swarm");
    if (!misfit) return fail(ctx, EMPSO_INVALID_ARG, "misfit is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    CK(ctx, launch_pso_step(ctx->pso, misfit, particles_out, st, rank));
    if (gbest_out) {
        CK(ctx, cudaMemcpyAsync(gbest_out, ctx->pso.gk, sizeof(int), cudaMemcpyDeviceToHost, st));
        CK(ctx, cudaStreamSynchronize(st));
    }
    return EMPSO_OK;
}

empso_status surrogate_init(empso_ctx *ctx, int32_t hidden, int32_t capacity, float lr, uint64_t seed)
{
    if (!ctx) return EMPSO_INVALID_ARG;
    ctx->err.clear();
    if (!ctx->has_pso) return fail(ctx, EMPSO_NOT_INITIALIZED, "the surrogate needs a swarm (its bounds)");
    if (ctx->has_sur) return fail(ctx, EMPSO_INVALID_ARG, "surrogate already initialised");
    if (hidden < 16 || hidden > 1024 || hidden % 16 || capacity < 1 || !(lr > 0))
        return fail(ctx, EMPSO_INVALID_ARG, "need 16 <= hidden <= 1024 (multiple of 16), capacity >= 1, lr > 0");
    SurDev &s = ctx->sur;
    const int K = ctx->pso.D, H = hidden, P = ctx->pso.P;
    s.K = K;
    s.H = H;
    s.cap = capacity;
    s.rows_max = std::max(P, 1024);
    s.off_W1 = 0;
    s.off_b1 = (long long)H * K;
    s.off_W2 = s.off_b1 + H;
    s.off_b2 = s.off_W2 + (long long)H * H;
    s.off_w3 = s.off_b2 + H;
    s.off_b3 = s.off_w3 + H;
    s.n_params = s.off_b3 + 1;
    s.lr = lr;
    s.seed = seed;
    s.xmin = ctx->pso.xmin;
    s.xmax = ctx->pso.xmax;
    auto alloc = [&](void **p, size_t bytes) {
        cudaError_t e = cudaMalloc(p, std::max<size_t>(bytes, 16));
        if (e == cudaSuccess) ctx->sur_mem.push_back(*p);
        return e;
    };
    const size_t R = s.rows_max;
    const size_t np = s.n_params;
    CK(ctx, alloc((void **)&s.p, 4 * np));
    CK(ctx, alloc((void **)&s.g, 4 * np));
    CK(ctx, alloc((void **)&s.m, 4 * np));
    CK(ctx, alloc((void **)&s.v, 4 * np));
    CK(ctx, alloc((void **)&s.W1b, 2 * (size_t)H * K));
    CK(ctx, alloc((void **)&s.W2b, 2 * (size_t)H * H));
    CK(ctx, alloc((void **)&s.Xb, 2 * R * K));
    CK(ctx, alloc((void **)&s.A1b, 2 * R * H));
    CK(ctx, alloc((void **)&s.dZb, 2 * R * H));
    CK(ctx, alloc((void **)&s.Z1, 4 * R * H));
    CK(ctx, alloc((void **)&s.Z2, 4 * R * H));
    CK(ctx, alloc((void **)&s.dZf, 4 * R * H));
    CK(ctx, alloc((void **)&s.dA, 4 * R * H));
    CK(ctx, alloc((void **)&s.y, 4 * R));
    CK(ctx, alloc((void **)&s.dy, 4 * R));
    CK(ctx, alloc((void **)&s.tb, 4 * R));
    CK(ctx, alloc((void **)&s.rows, 4 * R));
    CK(ctx, alloc((void **)&s.loss, 4));
    CK(ctx, alloc((void **)&s.stats, 8));
    CK(ctx, alloc((void **)&s.xbuf, 4 * (size_t)capacity * K));
    CK(ctx, alloc((void **)&s.ybuf, 4 * (size_t)capacity));
    CK(ctx, alloc((void **)&s.count, 4));
    CK(ctx, alloc((void **)&s.rho, 4));
    CK(ctx, alloc((void **)&ctx->sel_rows, 4 * (size_t)P));
    CK(ctx, alloc((void **)&ctx->xk, 4 * (size_t)P * K));
    CK(ctx, alloc((void **)&ctx->fk, 8 * (size_t)P));
    CK(ctx, alloc((void **)&ctx->fit_full, 8 * (size_t)P));
    CK(ctx, alloc((void **)&ctx->rank_full, 8 * (size_t)P));
    CK(ctx, alloc((void **)&ctx->logphi, 4 * (size_t)P));
    // He-uniform weights (limit sqrt(6 / fan_in)), zero biases, from the seed
    std::vector<float> h(np, 0.f);
    std::mt19937_64 rng(seed);
    std::uniform_real_distribution<double> u(-1.0, 1.0);
    const double l1 = std::sqrt(6.0 / K), l2 = std::sqrt(6.0 / H);
    for (long long i = 0; i < (long long)H * K; ++i) h[s.off_W1 + i] = (float)(l1 * u(rng));
    for (long long i = 0; i < (long long)H * H; ++i) h[s.off_W2 + i] = (float)(l2 * u(rng));
    for (long long i = 0; i < H; ++i) h[s.off_w3 + i] = (float)(l2 * u(rng));
    const float stats0[2] = {0.f, 1.f};
    CK(ctx, cudaMemcpy(s.p, h.data(), 4 * np, cudaMemcpyHostToDevice));
    CK(ctx, cudaMemset(s.m, 0, 4 * np));
    CK(ctx, cudaMemset(s.v, 0, 4 * np));
    CK(ctx, cudaMemset(s.count, 0, 4));
    CK(ctx, cudaMemset(s.rho, 0, 4));
    CK(ctx, cudaMemcpy(s.stats, stats0, 8, cudaMemcpyHostToDevice));
    CK(ctx, sur_refresh_bf16(s, 0));
    CK(ctx, sur_prepare_tc());
    s.tc = 1;
    s.err = ctx->dev_err;
    CK(ctx, cudaStreamCreateWithFlags(&ctx->sur_stream, cudaStreamNonBlocking));
    CK(ctx, cudaEventCreateWithFlags(&ctx->sur_fork, cudaEventDisableTiming));
    CK(ctx, cudaEventCreateWithFlags(&ctx->sur_done, cudaEventDisableTiming));
    CK(ctx, cudaDeviceSynchronize());
    ctx->has_sur = true;
    return EMPSO_OK;
}

#define NEED_SUR(ctx)                                                                   \
    do {                                                                                \
        if (!ctx) return EMPSO_INVALID_ARG;                                             \
        ctx->err.clear();                                                               \
        if (!ctx->has_sur) return fail(ctx, EMPSO_NOT_INITIALIZED, "no surrogate");      \
    } while (0)

// Every use of the network waits for training still running beside the
// modelling of the last prescreen generation.
#define JOIN_SUR(ctx, st)                                                               \
    do {                                                                                \
        if ((ctx)->sur_done_rec) CK(ctx, cudaStreamWaitEvent((st), (ctx)->sur_done, 0));  \
    } while (0)

empso_status surrogate_set_overlap(empso_ctx *ctx, int32_t enable)
{
    NEED_SUR(ctx);
    ctx->sur_overlap = enable != 0;
    return EMPSO_OK;
}

empso_status surrogate_set_policy(empso_ctx *ctx, int32_t recent, float min_rank_corr, int32_t patience)
{
    NEED_SUR(ctx);
    if (recent < 0 || !(min_rank_corr >= -1.f && min_rank_corr <= 1.f) || patience < 0)
        return fail(ctx, EMPSO_INVALID_ARG, "need recent >= 0, -1 <= min_rank_corr <= 1 and patience >= 0");
    ctx->sur.recent = recent;
    ctx->sur_rho_min = min_rank_corr;
    ctx->sur_patience = patience;
    ctx->sur_stall = 0;
    return EMPSO_OK;
}

empso_status surrogate_last_rank_corr(empso_ctx *ctx, float *rho, void *stream)
{
    NEED_SUR(ctx);
    if (!rho) return fail(ctx, EMPSO_INVALID_ARG, "null rho");
    cudaStream_t st = (cudaStream_t)stream;
    JOIN_SUR(ctx, st);
    CK(ctx, cudaMemcpyAsync(rho, ctx->sur.rho, sizeof(float), cudaMemcpyDeviceToHost, st));
    CK(ctx, cudaStreamSynchronize(st));
    return EMPSO_OK;
}

empso_status surrogate_set_backend(empso_ctx *ctx, int32_t kind)
{
    NEED_SUR(ctx);
    if (kind != 0 && kind != 1) return fail(ctx, EMPSO_INVALID_ARG, "backend must be 0 or 1");
    ctx->sur.tc = kind;
    return EMPSO_OK;
}

empso_status surrogate_predict(empso_ctx *ctx, const float *particles, int32_t P, float *logphi,
                               void *stream)
{
    NEED_SUR(ctx);
    JOIN_SUR(ctx, (cudaStream_t)stream);
    if (P < 0 || P > ctx->sur.rows_max || (P > 0 && (!particles || !logphi)))
        return fail(ctx, EMPSO_INVALID_ARG, "bad particles/logphi or too many rows");
    if (P == 0) return EMPSO_OK;
    CK(ctx, sur_predict(ctx->sur, particles, P, logphi, (cudaStream_t)stream));
    return EMPSO_OK;
}

empso_status surrogate_add(empso_ctx *ctx, const float *particles, const double *misfit, int32_t n,
                           void *stream)
{
    NEED_SUR(ctx);
    JOIN_SUR(ctx, (cudaStream_t)stream);
    if (n < 0 || (n > 0 && (!particles || !misfit))) return fail(ctx, EMPSO_INVALID_ARG, "bad particles/misfit");
    if (n == 0) return EMPSO_OK;
    CK(ctx, sur_append(ctx->sur, particles, misfit, nullptr, n, (cudaStream_t)stream));
    return EMPSO_OK;
}

empso_status surrogate_train(empso_ctx *ctx, int32_t steps, int32_t batch, void *stream)
{
    NEED_SUR(ctx);
    JOIN_SUR(ctx, (cudaStream_t)stream);
    if (steps < 0 || batch < 1 || batch > ctx->sur.rows_max)
        return fail(ctx, EMPSO_INVALID_ARG, "need steps >= 0 and 1 <= batch <= max rows");
    CK(ctx, sur_train(ctx->sur, steps, batch, (cudaStream_t)stream));
    return EMPSO_OK;
}

empso_status surrogate_params(empso_ctx *ctx, float *get, const float *set, int32_t *n_params,
                              void *stream)
{
    NEED_SUR(ctx);
    JOIN_SUR(ctx, (cudaStream_t)stream);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = 4 * (size_t)ctx->sur.n_params;
    if (n_params) *n_params = (int32_t)ctx->sur.n_params;
    if (get) CK(ctx, cudaMemcpyAsync(get, ctx->sur.p, bytes, cudaMemcpyDeviceToDevice, st));
    if (set) {
        CK(ctx, cudaMemcpyAsync(ctx->sur.p, set, bytes, cudaMemcpyDeviceToDevice, st));
        CK(ctx, sur_refresh_bf16(ctx->sur, st));
    }
    return EMPSO_OK;
}

empso_status surrogate_grad(empso_ctx *ctx, const float *particles, const float *target, int32_t n,
                            float *grad, float *loss, void *stream)
{
    NEED_SUR(ctx);
    JOIN_SUR(ctx, (cudaStream_t)stream);
    if (n < 1 || n > ctx->sur.rows_max || !particles || !target || !grad)
        return fail(ctx, EMPSO_INVALID_ARG, "bad particles/target/grad");
    cudaStream_t st = (cudaStream_t)stream;
    SurDev &s = ctx->sur;
    CK(ctx, sur_normalize(s, particles, nullptr, n, s.Xb, st));
    CK(ctx, sur_backward(s, s.Xb, target, n, loss ? loss : s.loss, st));
    CK(ctx, cudaMemcpyAsync(grad, s.g, 4 * (size_t)s.n_params, cudaMemcpyDeviceToDevice, st));
    return EMPSO_OK;
}

empso_status surrogate_generation(empso_ctx *ctx, const empso_shot *shots, int32_t S,
                                  const float *d_obs, double keep_frac, int32_t warm,
                                  int32_t train_steps, int32_t batch, double *misfit_out,
                                  int32_t *n_modelled, void *stream)
{
    NEED_SUR(ctx);
    if (!d_obs || !(keep_frac > 0 && keep_frac <= 1) || train_steps < 0 || batch < 1 ||
        batch > ctx->sur.rows_max)
        return fail(ctx, EMPSO_INVALID_ARG, "bad d_obs, keep fraction or training settings");
    empso_status rc = check_shots(ctx, shots, S, -1);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    SurDev &s = ctx->sur;
    const int P = ctx->pso.P, K = ctx->pso.D;
    for (int i = 0; i < S; ++i) {
        if (ctx->grids[shots[i].grid_id].dev.K != K)
            return fail(ctx, EMPSO_INVALID_ARG, "swarm dimension differs from the grids' control nodes");
    }
    JOIN_SUR(ctx, st);
    // how many pairs the replay buffer holds (host read: decides the branch)
    int have = 0;
    float rho = 1.f;
    int gk[2] = {0, 0};
    CK(ctx, cudaMemcpyAsync(&have, s.count, sizeof(int), cudaMemcpyDeviceToHost, st));
    if (ctx->sur_rho_min > 0.f && ctx->sur_screened)
        CK(ctx, cudaMemcpyAsync(&rho, s.rho, sizeof(float), cudaMemcpyDeviceToHost, st));
    if (ctx->sur_patience > 0) CK(ctx, cudaMemcpyAsync(gk, ctx->pso.gk, sizeof gk, cudaMemcpyDeviceToHost, st));
    CK(ctx, cudaStreamSynchronize(st));
    // stagnation: pre-screened generations in a row after which the swarm's
    // best misfit (its global best) did not improve
    if (ctx->sur_patience > 0) {
        double best = HUGE_VAL;
        CK(ctx, cudaMemcpyAsync(&best, ctx->pso.pf + gk[0], sizeof best, cudaMemcpyDeviceToHost, st));
        CK(ctx, cudaStreamSynchronize(st));
        ctx->sur_stall = ctx->sur_screened && !(best < ctx->sur_best) ? ctx->sur_stall + 1 : 0;
        ctx->sur_best = best;
    }
    if ((rc = strict_begin(ctx, st))) return rc;
    Models mod;
    int k;
    // the whole swarm is modelled while the buffer warms up, after a
    // pre-screened generation whose predictions ranked the modelled particles
    // too poorly (rank correlation below the policy's minimum), and after
    // `patience` pre-screened generations in a row without a new best
    const bool stalled = ctx->sur_patience > 0 && ctx->sur_stall >= ctx->sur_patience;
    const bool fallback = (ctx->sur_rho_min > 0.f && ctx->sur_screened && rho < ctx->sur_rho_min) || stalled;
    if (stalled) ctx->sur_stall = 0;
    ctx->sur_screened = false;
    if (have < warm || fallback) {
        // warm-up: model every particle, then train on everything so far
        k = P;
        mod.particles = ctx->xf;
        mod.M = P;
        if ((rc = run_batch(ctx, mod, shots, S, d_obs, nullptr, ctx->fit_full, st))) return rc;
        CK(ctx, sur_append(s, ctx->xf, ctx->fit_full, nullptr, P, st));
        CK(ctx, sur_train(s, train_steps, batch, st));
        CK(ctx, launch_pso_step(ctx->pso, ctx->fit_full, nullptr, st, nullptr));
    } else {
        // pre-screen: model the keep_frac fraction with the smallest predictions
        k = std::max(1, (int)std::lround(keep_frac * P));
        CK(ctx, sur_predict(s, ctx->xf, P, ctx->logphi, st));
        CK(ctx, sur_select(ctx->logphi, P, k, ctx->sel_rows, st));
        CK(ctx, sur_gather(ctx->xf, ctx->sel_rows, k, K, ctx->xk, st));
        // overlap mode: training on the pairs of the earlier generations (the
        // first `have` rows) runs on a second stream beside this generation's
        // modelling, which appends only behind those rows; when the append
        // would wrap the ring onto them it runs first instead (same data,
        // same result).  Default: train after the append, on every pair.  The
        // modelling is enqueued before the training's many small launches, so
        // that the GPU starts on it while the host is still issuing them.
        const bool beside = train_steps > 0 && ctx->sur_overlap && (long long)have + k <= s.cap;
        if (train_steps > 0 && ctx->sur_overlap && !beside) CK(ctx, sur_train(s, train_steps, batch, st, have));
        // the training's fork is recorded once the model fields are written,
        // just before the modelling launch
        mod.particles = ctx->xk;
        mod.M = k;
        if ((rc = run_batch(ctx, mod, shots, S, d_obs, nullptr, ctx->fk, st, beside ? ctx->sur_fork : nullptr)))
            return rc;
        if (beside) {
            CK(ctx, cudaStreamWaitEvent(ctx->sur_stream, ctx->sur_fork, 0));
            CK(ctx, sur_train(s, train_steps, batch, ctx->sur_stream, have));
            CK(ctx, cudaEventRecord(ctx->sur_done, ctx->sur_stream));
            ctx->sur_done_rec = true;
        }
        CK(ctx, sur_rank_corr(ctx->fk, ctx->sel_rows, ctx->logphi, k, s.rho, st));
        ctx->sur_screened = true;
        CK(ctx, sur_append(s, ctx->xk, ctx->fk, nullptr, k, st));
        CK(ctx, sur_scatter(ctx->sel_rows, ctx->fk, k, ctx->logphi, P, ctx->fit_full, ctx->rank_full, st));
        if (train_steps > 0 && !ctx->sur_overlap) CK(ctx, sur_train(s, train_steps, batch, st));
        CK(ctx, launch_pso_step(ctx->pso, ctx->fit_full, nullptr, st, ctx->rank_full));
    }
    if (misfit_out)
        CK(ctx, cudaMemcpyAsync(misfit_out, ctx->fit_full, sizeof(double) * P, cudaMemcpyDeviceToDevice, st));
    if (n_modelled) *n_modelled = k;
    return strict_end(ctx, EMPSO_OK, st);
}

empso_status empso_set_strict(empso_ctx *ctx, int32_t enable)
{
    if (!ctx) return EMPSO_INVALID_ARG;
    ctx->err.clear();
    ctx->strict = enable != 0;
    return EMPSO_OK;
}

empso_status empso_nonfinite_count(empso_ctx *ctx, int64_t *count, int32_t reset, void *stream)
{
    if (!ctx) return EMPSO_INVALID_ARG;
    ctx->err.clear();
    if (!count) return fail(ctx, EMPSO_INVALID_ARG, "count is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    unsigned long long n = 0;
    CK(ctx, cudaMemcpyAsync(&n, ctx->nonfinite, sizeof n, cudaMemcpyDeviceToHost, st));
    CK(ctx, cudaStreamSynchronize(st));
    if (reset) CK(ctx, cudaMemsetAsync(ctx->nonfinite, 0, sizeof n, st));
    *count = (int64_t)n;
    return EMPSO_OK;
}

// ---------------------------------------------------------------------------
// Checkpoints.  File layout (native byte order, no padding):
//   "EMPSOCK1" | u32 version | u32 parts (1 swarm, 2 surrogate)
//   swarm:     i32 P, D | u64 seed | i32 g, k | f64 xmin[D], xmax[D]
//              | f64 x[P D], v[P D], p[P D], pf[P] | i32 order[P]
//   surrogate: i32 K, H, cap | u64 seed | i32 t, sample_step, count
//              | i32 screened | f32 rank correlation of that generation
//              | i32 stalled generations | f64 best misfit of the stall count
//              | f32 stats[2] | f32 params[n], m[n], v[n]
//              | f32 xbuf[rows K], ybuf[rows] with rows = min(count, cap)
//   u64 FNV-1a hash of every preceding byte
// ---------------------------------------------------------------------------
}  // extern "C"

namespace {

const char CK_MAGIC[8] = {'E', 'M', 'P', 'S', 'O', 'C', 'K', '1'};
constexpr uint32_t CK_VERSION = 3;

uint64_t fnv1a(const unsigned char *p, size_t n)
{
    uint64_t h = 1469598103934665603ull;
    for (size_t i = 0; i < n; ++i) {
        h ^= p[i];
        h *= 1099511628211ull;
    }
    return h;
}

struct CkOut {
    std::vector<unsigned char> b;
    void put(const void *p, size_t n)
    {
        const unsigned char *c = (const unsigned char *)p;
        b.insert(b.end(), c, c + n);
    }
    template <class T> void val(T v) { put(&v, sizeof v); }
};

struct CkIn {
    const std::vector<unsigned char> &b;
    size_t pos = 0;
    bool get(void *p, size_t n)
    {
        if (n > b.size() - pos) return false;
        memcpy(p, b.data() + pos, n);
        pos += n;
        return true;
    }
    template <class T> bool val(T &v) { return get(&v, sizeof v); }
};

// append n elements of device array d to the checkpoint
template <class T> cudaError_t dev_put(CkOut &o, const T *d, size_t n)
{
    std::vector<T> h(n);
    cudaError_t e = n ? cudaMemcpy(h.data(), d, n * sizeof(T), cudaMemcpyDeviceToHost) : cudaSuccess;
    if (e == cudaSuccess) o.put(h.data(), n * sizeof(T));
    return e;
}

}  // namespace

extern "C" {

empso_status empso_save(empso_ctx *ctx, const char *path)
{
    if (!ctx) return EMPSO_INVALID_ARG;
    ctx->err.clear();
    if (!path || !*path) return fail(ctx, EMPSO_INVALID_ARG, "path is empty");
    if (!ctx->has_pso) return fail(ctx, EMPSO_NOT_INITIALIZED, "context has no swarm to save");
    CK(ctx, cudaDeviceSynchronize());
    CkOut o;
    o.put(CK_MAGIC, 8);
    o.val<uint32_t>(CK_VERSION);
    o.val<uint32_t>(1u | (ctx->has_sur ? 2u : 0u));
    const PsoDev &q = ctx->pso;
    const size_t PD = (size_t)q.P * q.D;
    int gk[2];
    CK(ctx, cudaMemcpy(gk, q.gk, sizeof gk, cudaMemcpyDeviceToHost));
    o.val<int32_t>(q.P);
    o.val<int32_t>(q.D);
    o.val<uint64_t>(q.seed);
    o.val<int32_t>(gk[0]);
    o.val<int32_t>(gk[1]);
    CK(ctx, dev_put(o, q.xmin, q.D));
    CK(ctx, dev_put(o, q.xmax, q.D));
    CK(ctx, dev_put(o, q.x, PD));
    CK(ctx, dev_put(o, q.v, PD));
    CK(ctx, dev_put(o, q.p, PD));
    CK(ctx, dev_put(o, q.pf, (size_t)q.P));
    CK(ctx, dev_put(o, q.order, (size_t)q.P));
    if (ctx->has_sur) {
        const SurDev &s = ctx->sur;
        int count = 0;
        CK(ctx, cudaMemcpy(&count, s.count, sizeof count, cudaMemcpyDeviceToHost));
        const size_t rows = (size_t)std::min(count, s.cap);
        o.val<int32_t>(s.K);
        o.val<int32_t>(s.H);
        o.val<int32_t>(s.cap);
        o.val<uint64_t>(s.seed);
        o.val<int32_t>(s.t);
        o.val<int32_t>(s.sample_step);
        o.val<int32_t>(count);
        float rho = 0.f;
        CK(ctx, cudaMemcpy(&rho, s.rho, sizeof rho, cudaMemcpyDeviceToHost));
        o.val<int32_t>(ctx->sur_screened ? 1 : 0);
        o.val<float>(rho);
        o.val<int32_t>(ctx->sur_stall);
        o.val<double>(ctx->sur_best);
        CK(ctx, dev_put(o, s.stats, 2));
        CK(ctx, dev_put(o, s.p, (size_t)s.n_params));
        CK(ctx, dev_put(o, s.m, (size_t)s.n_params));
        CK(ctx, dev_put(o, s.v, (size_t)s.n_params));
        CK(ctx, dev_put(o, s.xbuf, rows * s.K));
        CK(ctx, dev_put(o, s.ybuf, rows));
    }
    o.val<uint64_t>(fnv1a(o.b.data(), o.b.size()));
    // write beside the target and rename, so a crash never leaves half a file
    const std::string tmp = std::string(path) + ".tmp";
    FILE *f = fopen(tmp.c_str(), "wb");
    if (!f) return fail(ctx, EMPSO_IO_ERROR, "cannot open " + tmp + " for writing");
    const bool ok = fwrite(o.b.data(), 1, o.b.size(), f) == o.b.size();
    if ((fclose(f) != 0) || !ok) {
        remove(tmp.c_str());
        return fail(ctx, EMPSO_IO_ERROR, "short write to " + tmp);
    }
    if (rename(tmp.c_str(), path) != 0) {
        remove(tmp.c_str());
        return fail(ctx, EMPSO_IO_ERROR, std::string("cannot rename onto ") + path);
    }
    return EMPSO_OK;
}

empso_status empso_load(empso_ctx *ctx, const char *path)
{
    if (!ctx) return EMPSO_INVALID_ARG;
    ctx->err.clear();
    if (!path || !*path) return fail(ctx, EMPSO_INVALID_ARG, "path is empty");
    if (!ctx->has_pso) return fail(ctx, EMPSO_NOT_INITIALIZED, "context has no swarm to restore");
    std::vector<unsigned char> b;
    {
        FILE *f = fopen(path, "rb");
        if (!f) return fail(ctx, EMPSO_IO_ERROR, std::string("cannot open ") + path);
        unsigned char buf[1 << 16];
        size_t n;
        while ((n = fread(buf, 1, sizeof buf, f)) > 0) b.insert(b.end(), buf, buf + n);
        const bool bad = ferror(f) != 0;
        fclose(f);
        if (bad) return fail(ctx, EMPSO_IO_ERROR, std::string("read error on ") + path);
    }
    const auto corrupt = [&](const char *what) {
        return fail(ctx, EMPSO_IO_ERROR, std::string("not a valid checkpoint (") + what + "): " + path);
    };
    if (b.size() < 8 + 8 + 8) return corrupt("too short");
    uint64_t stored;
    memcpy(&stored, b.data() + b.size() - 8, 8);
    if (stored != fnv1a(b.data(), b.size() - 8)) return corrupt("checksum");
    b.resize(b.size() - 8);
    CkIn in{b};
    char magic[8];
    uint32_t version = 0, parts = 0;
    if (!in.get(magic, 8) || memcmp(magic, CK_MAGIC, 8) != 0) return corrupt("magic");
    if (!in.val(version) || version != CK_VERSION) return corrupt("version");
    if (!in.val(parts) || !(parts & 1u)) return corrupt("parts");
    const PsoDev &q = ctx->pso;
    int32_t P, D, g, k;
    uint64_t seed;
    if (!in.val(P) || !in.val(D) || !in.val(seed) || !in.val(g) || !in.val(k)) return corrupt("swarm header");
    if (P != q.P || D != q.D || seed != q.seed)
        return fail(ctx, EMPSO_INVALID_ARG, "checkpoint swarm (P, D, seed) differs from this context's");
    if (g < 0 || g >= P || k < 0) return corrupt("swarm g, k");
    const size_t PD = (size_t)P * D;
    std::vector<double> lo(D), hi(D), x(PD), v(PD), pp(PD), pf(P);
    std::vector<int32_t> order(P);
    if (!in.get(lo.data(), 8 * lo.size()) || !in.get(hi.data(), 8 * hi.size()) ||
        !in.get(x.data(), 8 * PD) || !in.get(v.data(), 8 * PD) || !in.get(pp.data(), 8 * PD) ||
        !in.get(pf.data(), 8 * pf.size()) || !in.get(order.data(), 4 * order.size()))
        return corrupt("swarm arrays");
    {
        std::vector<double> clo(D), chi(D);
        CK(ctx, cudaMemcpy(clo.data(), q.xmin, 8 * (size_t)D, cudaMemcpyDeviceToHost));
        CK(ctx, cudaMemcpy(chi.data(), q.xmax, 8 * (size_t)D, cudaMemcpyDeviceToHost));
        if (memcmp(clo.data(), lo.data(), 8 * (size_t)D) || memcmp(chi.data(), hi.data(), 8 * (size_t)D))
            return fail(ctx, EMPSO_INVALID_ARG, "checkpoint search bounds differ from this context's");
    }
    // surrogate part: validated in full before anything is written
    int32_t sK = 0, sH = 0, scap = 0, st_t = 0, st_step = 0, count = 0, screened = 0, stall = 0;
    uint64_t sseed = 0;
    double sbest = HUGE_VAL;
    float stats[2], rho = 0.f;
    std::vector<float> sp, sm, sv, xb, yb;
    const bool file_sur = (parts & 2u) != 0;
    if (file_sur) {
        if (!ctx->has_sur)
            return fail(ctx, EMPSO_NOT_INITIALIZED, "checkpoint holds a surrogate; call surrogate_init first");
        const SurDev &s = ctx->sur;
        if (!in.val(sK) || !in.val(sH) || !in.val(scap) || !in.val(sseed) || !in.val(st_t) ||
            !in.val(st_step) || !in.val(count) || !in.val(screened) || !in.val(rho) || !in.val(stall) ||
            !in.val(sbest) || !in.get(stats, sizeof stats))
            return corrupt("surrogate header");
        if (sK != s.K || sH != s.H || scap != s.cap)
            return fail(ctx, EMPSO_INVALID_ARG, "checkpoint surrogate (K, H, capacity) differs from this context's");
        if (count < 0 || st_t < 0 || st_step < 0 || (screened != 0 && screened != 1) || stall < 0)
            return corrupt("surrogate counters");
        const size_t np = (size_t)s.n_params, rows = (size_t)std::min(count, scap);
        sp.resize(np);
        sm.resize(np);
        sv.resize(np);
        xb.resize(rows * sK);
        yb.resize(rows);
        if (!in.get(sp.data(), 4 * np) || !in.get(sm.data(), 4 * np) || !in.get(sv.data(), 4 * np) ||
            !in.get(xb.data(), 4 * xb.size()) || !in.get(yb.data(), 4 * yb.size()))
            return corrupt("surrogate arrays");
    }
    if (in.pos != b.size()) return corrupt("trailing bytes");
    CK(ctx, cudaDeviceSynchronize());
    CK(ctx, cudaMemcpy(q.x, x.data(), 8 * PD, cudaMemcpyHostToDevice));
    CK(ctx, cudaMemcpy(q.v, v.data(), 8 * PD, cudaMemcpyHostToDevice));
    CK(ctx, cudaMemcpy(q.p, pp.data(), 8 * PD, cudaMemcpyHostToDevice));
    CK(ctx, cudaMemcpy(q.pf, pf.data(), 8 * (size_t)P, cudaMemcpyHostToDevice));
    CK(ctx, cudaMemcpy(q.order, order.data(), 4 * (size_t)P, cudaMemcpyHostToDevice));
    const int gk[2] = {g, k};
    CK(ctx, cudaMemcpy(q.gk, gk, sizeof gk, cudaMemcpyHostToDevice));
    CK(ctx, launch_xf_from_x(q, 0));
    if (file_sur) {
        SurDev &s = ctx->sur;
        CK(ctx, cudaMemcpy(s.p, sp.data(), 4 * sp.size(), cudaMemcpyHostToDevice));
        CK(ctx, cudaMemcpy(s.m, sm.data(), 4 * sm.size(), cudaMemcpyHostToDevice));
        CK(ctx, cudaMemcpy(s.v, sv.data(), 4 * sv.size(), cudaMemcpyHostToDevice));
        CK(ctx, cudaMemcpy(s.stats, stats, sizeof stats, cudaMemcpyHostToDevice));
        CK(ctx, cudaMemcpy(s.count, &count, sizeof count, cudaMemcpyHostToDevice));
        CK(ctx, cudaMemcpy(s.rho, &rho, sizeof rho, cudaMemcpyHostToDevice));
        ctx->sur_screened = screened != 0;
        ctx->sur_stall = stall;
        ctx->sur_best = sbest;
        if (!xb.empty()) {
            CK(ctx, cudaMemcpy(s.xbuf, xb.data(), 4 * xb.size(), cudaMemcpyHostToDevice));
            CK(ctx, cudaMemcpy(s.ybuf, yb.data(), 4 * yb.size(), cudaMemcpyHostToDevice));
        }
        s.seed = sseed;
        s.t = st_t;
        s.sample_step = st_step;
        CK(ctx, sur_refresh_bf16(s, 0));
    }
    CK(ctx, cudaDeviceSynchronize());
    return EMPSO_OK;
}

}  // extern "C"
