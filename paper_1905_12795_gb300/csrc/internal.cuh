// Internal declarations shared by the translation units of the EMPSO CUDA
// library.  Not part of the public ABI (include/empso.h is).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "empso.h"

namespace empso {

// Every wavefield / model buffer carries HALO zero cells around the padded
// grid on all sides, enough for the widest stencil (space order 16, radius 8),
// so the stencil never tests bounds.  Padded node (I, J) lives at
// buf[(J + HALO) * pitch + I + HALO]; the interior starts 32 bytes into a row,
// so float4 group q (nodes 4q .. 4q+3) is 16-byte aligned and sits at float4
// index HALO4 + q of its row.
constexpr int HALO = 8;
constexpr int HALO4 = HALO / 4;
constexpr int MAX_R = 8;
// radius of the widest stencil of the cluster and streaming modelling kernels
// (orders 2, 4, 8); order 16 runs on the plain streaming kernel and the
// per-step adjoint kernels
constexpr int MAX_R_FAST = 4;
constexpr int MAX_PSO_P = 2048;
constexpr int MAX_PSO_D = 1024;

// Wall-clock limit of every device-side wait (mbarrier phases): a wait that
// runs past it records EMPSO_TIMEOUT in the context's status word instead of
// spinning on.
constexpr unsigned long long WAIT_LIMIT_NS = 1000000000ull;

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
    return t;
}

// Device-side description of one modelling grid.
struct GridDev {
    int nx, nz, pad, R;      // physical nodes, damping cells, stencil radius
    int NX, NZ;              // padded grid
    int NQ;                  // float4 groups per row = ceil(NX / 4)
    int pitch;               // floats per buffer row (multiple of 32)
    int rows;                // NZ + 2 HALO
    int nt;                  // time steps = trace samples
    int kx, kz, mode;        // control nodes and interpolation mode (2: level grid)
    int K;                   // control nodes per particle (kx kz, or the level grid's count)
    float water_z, v_water;  // fixed water layer: depth <= water_z (when > 0) takes v_water
    float dt, hx, hz;
    float vmin, vmax;
    float c[MAX_R + 1];      // centred 2nd-derivative weights c_0..c_R
    float cxm[MAX_R + 1];    // c_m / hx^2 (m >= 1), [0] = c_0 (1/hx^2 + 1/hz^2)
    float czm[MAX_R + 1];    // c_m / hz^2 (m >= 1), [0] = 0
    float cres;              // (c_0 + 2 c_1 + 2 c_2)(1/hx^2 + 1/hz^2): the centre weight left
                             // once the m = 1, 2 terms are taken as differences (stencil.cuh)
    const float *wavelet;    // [nt]      Ricker r(n dt)
    const float *ex;         // [pitch]   eta_x dt / 2 per buffer column (0 in halo)
    const float *ez;         // [rows]    eta_z dt / 2 per buffer row (0 in halo)
    const float *Wx;         // [nx][kx]  interpolation weights along x
    const float *Wz;         // [nz][kz]  interpolation weights along z
    const int4 *lidx;        // [nz][nx]  level grid: the four nodes of each point
    const float4 *lw;        // [nz][nx]  and their weights
    long long field;         // floats per buffer = rows * pitch
};

// One (model, shot) modelling instance of a launch.
struct Inst {
    const float *a;          // model field v^2 dt^2, buffer layout of the grid
    const float *dobs;       // [nt][nrec] observed traces, or null
    float *traces;           // [nt][nrec] output traces, or null
    const float2 *rec;       // receiver positions (m) of this shot
    int grid;                // index into the grid table
    int nrec;
    float sx, sz;            // source position (m)
    int out;                 // slot of the partial misfit
    int run;                 // on-chip kernel: rows per run for this instance (0: the launch's)
    float *hist;             // [nt + 1][field] gradient history (L u^n into slot n + 1,
                             // buffer layout), or null; the HIST variants of the cluster
                             // kernels only
};

// Centred 2nd-derivative weights c_0..c_R of space order `order` (false when
// the order is not supported).
bool fd_weights(int order, double *c, int *R);
// Validate a grid description and derive its host-side part (stencil
// weights, time axis, buffer layout); the device table pointers stay null.
// Returns EMPSO_INVALID_ARG / EMPSO_UNSUPPORTED with a message in `err`.
empso_status derive_grid(const empso_grid &s, int id, GridDev &g, std::string &err);

// Host-side launchers (each enqueues on `st`).  Return cudaSuccess or the
// launch error.
cudaError_t launch_grid_tables(const GridDev &g, float *ex, float *ez, float *wavelet,
                               float *Wx, float *Wz, double vmax_damp, double f0,
                               cudaStream_t st);
// Adjoint-state gradient (adjoint.cu): one (model, shot) instance.
struct AdjInst {
    const float *a;      // model field a = v^2 dt^2 (buffer layout)
    const float *B;      // f a, f = 1 / (1 + t)
    float *H;            // history [nt + 1][field]: H[n + 1] = L u^n (H[0] unused)
    float *mu;           // adjoint fields [4][field]: slot k mod 4 (two-step backward) or k mod 2
    float *G;            // dphi/da of this shot [field]
    float *J;            // receiver terms w R^T e of adjoint steps [4][field] (slot k mod 4), zero elsewhere
    float *E;            // residuals [nt][nrec]
    const float *dobs;   // [nt][nrec]
    const float2 *rec;   // receiver positions
    int nrec;
    float sx, sz, w;     // source position, shot weight
    int jr0, jr1;        // padded rows that may hold a receiver term (J is zero elsewhere)
};
cudaError_t launch_adj_prep(const GridDev &g, const float *a, float *B, int M, cudaStream_t st);
// the per-step forward pass: the time levels live in two of each instance's
// adjoint slots (zeroed before; u^{n+1} overwrites u^{n-1}) and the history
// takes L u^n in slot n + 1
cudaError_t launch_adj_forward(const GridDev &g, const AdjInst *insts, int n_inst, int rec_threads,
                               cudaStream_t st);
// e = d - d_obs in place in every instance's E (after an on-chip forward pass
// that wrote its traces there)
cudaError_t launch_adj_residual(const GridDev &g, const AdjInst *insts, int n_inst, int rec_max,
                                cudaStream_t st);
// the backward pass of instances insts[0 .. n_inst), one of several chains
// that together run n_all instances at once; the history holds L u^n in slot
// n + 1
cudaError_t launch_adj_backward(const GridDev &g, const AdjInst *insts, int n_inst, int n_all, int rec_threads,
                                cudaStream_t st);
// T: scratch of max(M * NZ * nx floats, M * S * 64 doubles), 8-byte aligned
// (the misfit partials, then the x-folded gradient)
cudaError_t launch_adj_finish(const GridDev &g, const AdjInst *insts, int M, int S, const float *vel,
                              double *phi, double *misfit, float *grad, float *T, cudaStream_t st);
// the misfit of every model from the residuals of a forward pass (part:
// scratch of M * S * 64 doubles)
cudaError_t launch_adj_misfit(const GridDev &g, const AdjInst *insts, int M, int S, double *phi,
                              double *misfit, double *part, cudaStream_t st);
cudaError_t launch_fwi_step(const float *v, const float *g, float alpha, float vmin, float vmax,
                            float *out, int n, cudaStream_t st);
cudaError_t launch_fwi_dots(const float *a, const float *b, const float *c, const float *d, int n,
                            double *r, cudaStream_t st);

// L2-resident cluster variant (wave_l2.cu): time levels in a per-cluster
// global buffer of l2_slot_f4 float4 each.
int l2_max_threads();
size_t l2_smem_bytes(int ring_pitch);
long long l2_slot_f4(const GridDev &g, int C);
bool l2_fits(const GridDev &g, int C);
cudaError_t l2_configure(int R, size_t smem, int C);
// clusters of the modelling (hist = false) or history (hist = true) instantiation
// that fit the device at once
int l2_max_clusters(int R, int C, int threads, size_t smem, bool hist = false);
cudaError_t launch_wave_l2(int R, const GridDev *grids_dev, const Inst *insts, int n_inst, int *counter,
                           int C, int n_clusters, int threads, float4 *slots, long long slot_f4,
                           int ring_pitch, size_t smem, double *partial, cudaStream_t st, bool hist = false);

// Band-limited resampling of traces (filter.cu).
long long lowpass_span(double dt_in, double dt_out, double W);
size_t lowpass_smem_bytes(long long span);
cudaError_t lowpass_configure(size_t smem);
cudaError_t launch_lowpass(const float *in, int S, int nt_in, int nrec, double dt_in, float *out,
                           int nt_out, double dt_out, double fc, double W, size_t smem,
                           cudaStream_t st);

cudaError_t launch_level_taps(const GridDev &g, int L, const float *level_z, const int *level_off,
                              const float *node_x, int4 *lidx, float4 *lw, cudaStream_t st);
cudaError_t launch_interp(const GridDev &g, const float *particles, int P, float *a_fields,
                          long long field_stride, float *vel_out, cudaStream_t st);
cudaError_t launch_vel_to_field(const GridDev &g, const float *vel, int M, float *a_fields,
                                long long field_stride, cudaStream_t st);
cudaError_t launch_wave(const GridDev *grids_dev, const Inst *insts, int n_inst,
                        int *counter, float *slots, long long slot_floats, int n_ctas,
                        int threads, double *partial, cudaStream_t st);
cudaError_t launch_finalize(const double *partial, const float *weights, int P, int S,
                            double *misfit, unsigned long long *nf, cudaStream_t st);
int wave_max_ctas_per_sm(int threads);

// On-chip variant (wave_resident.cu): one thread-block cluster per instance.
// float4 per slab row of its damping table: one for the column groups outside
// the x-damping layer and one per group with a lane in it
__host__ __device__ inline int resident_gtab_width(const GridDev &g)
{
    const int qa = g.NQ < (g.pad + 3) / 4 ? g.NQ : (g.pad + 3) / 4;
    int qb = (g.NX - g.pad) / 4;
    qb = qb > g.NQ ? g.NQ : qb;
    qb = qb < qa ? qa : qb;
    return 1 + qa + (g.NQ - qb);
}
// `rows`: the rows-per-thread shape (8 or 13).
int resident_max_threads(int rows);
int resident_default_rows();
bool resident_rows_supported(int rows);
int resident_grid_run(const GridDev &g, int Ce, int threads, int rows);
int resident_threads(const GridDev &g, int C, int rows);
size_t resident_smem_bytes(const GridDev &g, int C, int ring_pitch);
bool resident_fits(const GridDev &g, int C, int ring_pitch, size_t smem_limit, int rows);
cudaError_t resident_configure(int R, size_t smem_bytes, int C);
// clusters of the modelling (hist = false) or history instantiation that fit at once
int resident_max_clusters(int R, int C, int threads, size_t smem_bytes, int rows, bool hist = false);
// `hist`: the variant that also streams every u^{n+1} into Inst::hist (no
// halved units)
cudaError_t launch_wave_resident(int R, const GridDev *grids_dev, const Inst *insts, const int4 *units,
                                 int n_units, bool pairs, int *counter, int C, int n_clusters, int threads,
                                 int rows, int ring_pitch, size_t smem_bytes, double *partial,
                                 cudaStream_t st, bool hist = false);

// TMA-pipelined streaming variant (wave_stream.cu).
int stream_max_threads();
size_t stream_smem_bytes(int R, int pitch, int rec_max);
cudaError_t stream_configure(int R, size_t smem);
cudaError_t launch_wave_stream(int R, const GridDev *grids_dev, const Inst *insts, int n_inst,
                               int *counter, float *slots, long long slot_floats, int n_ctas,
                               int threads, size_t smem, int rec_max, int *err, double *partial,
                               cudaStream_t st);

// Message returned by empso_last_error(NULL) for calls made without a context.
void set_global_error(const char *msg);

// Swarm state on the device.
struct PsoDev {
    int P, D, NM, em_start, em_enabled;
    double c1, c2, lambda, p_em;
    uint64_t seed;
    const double *xmin, *xmax;   // [D]
    double *x, *v, *p;           // [P][D]
    double *pf;                  // [P]
    int *order;                  // [P]
    int *gk;                     // {g, k}
    int *rank_of;                // [P] EM rank of each particle in the current step
    float *xf;                   // [P][D] float copy of x (what generations evaluate)
};
cudaError_t launch_pso_init(const PsoDev &s, float *particles_out, cudaStream_t st);
cudaError_t launch_pso_step(const PsoDev &s, const double *misfit, float *particles_out,
                            cudaStream_t st, const double *rank = nullptr);
cudaError_t launch_xf_from_x(const PsoDev &s, cudaStream_t st);

// Surrogate network (surrogate.cu): flat FP32 parameters in the order
// W1 [H][K], b1 [H], W2 [H][H], b2 [H], w3 [H], b3 [1]; BF16 copies of W1, W2.
struct SurDev {
    int K = 0, H = 0, cap = 0, rows_max = 0;
    long long n_params = 0, off_W1 = 0, off_b1 = 0, off_W2 = 0, off_b2 = 0, off_w3 = 0, off_b3 = 0;
    float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
    __nv_bfloat16 *W1b = nullptr, *W2b = nullptr;
    const double *xmin = nullptr, *xmax = nullptr;
    __nv_bfloat16 *Xb = nullptr, *A1b = nullptr, *dZb = nullptr;
    float *Z1 = nullptr, *Z2 = nullptr, *y = nullptr, *dy = nullptr, *dZf = nullptr, *dA = nullptr;
    float *tb = nullptr, *loss = nullptr, *stats = nullptr;
    int *rows = nullptr;
    float *xbuf = nullptr, *ybuf = nullptr;
    int *count = nullptr;
    uint64_t seed = 0;
    int sample_step = 0, t = 0;
    int recent = 0;          // > 0: half of every minibatch from the newest `recent` pairs
    float *rho = nullptr;    // Spearman correlation of predicted and true misfits of the
                             // last pre-screened generation's modelled particles
    float lr = 1e-3f, beta1 = 0.9f, beta2 = 0.999f, eps = 1e-8f;
    int tc = 1;              // dense layers: 1 = tcgen05 (TMEM accumulator), 0 = mma.sync
    int *err = nullptr;      // status word for a tcgen05 completion wait that gives up
};
cudaError_t sur_forward(const SurDev &s, const __nv_bfloat16 *Xb, int n, float *y, cudaStream_t st);
cudaError_t sur_backward(const SurDev &s, const __nv_bfloat16 *Xb, const float *t, int n, float *loss,
                         cudaStream_t st);
cudaError_t sur_adam(SurDev &s, cudaStream_t st);
cudaError_t sur_refresh_bf16(const SurDev &s, cudaStream_t st);
cudaError_t sur_normalize(const SurDev &s, const float *x, const int *rows, int n, __nv_bfloat16 *out,
                          cudaStream_t st);
cudaError_t sur_predict(const SurDev &s, const float *x, int n, float *logphi, cudaStream_t st);
cudaError_t sur_append(const SurDev &s, const float *x, const double *misfit, const int *rows, int n,
                       cudaStream_t st);
// have >= 0: train on the first min(have, cap) replay rows (a host snapshot);
// have < 0: on the rows the device count says are filled
cudaError_t sur_train(SurDev &s, int steps, int B, cudaStream_t st, int have = -1);
cudaError_t sur_select(const float *key, int P, int k, int *rows, cudaStream_t st);
// rank correlation of fk[j] (true misfits of the k modelled particles) with
// logphi[rows[j]] (their predictions) into *rho (one block)
cudaError_t sur_rank_corr(const double *fk, const int *rows, const float *logphi, int k, float *rho,
                          cudaStream_t st);
cudaError_t sur_prepare_tc();
cudaError_t sur_gather(const float *x, const int *rows, int k, int K, float *out, cudaStream_t st);
cudaError_t sur_scatter(const int *rows, const double *fk, int k, const float *logphi, int P,
                        double *fit, double *rank, cudaStream_t st);

}  // namespace empso
