// Adjoint-state gradient of the l2 misfit with respect to the velocity model
// (the local full-waveform inversion of section "Testing approach": steepest
// descent on the misfit's gradient, started from the EMPSO model).
//
// Forward scheme (the modelling kernels' scheme, written per point):
//   u^{n+1} = 2 f u^n - g u^{n-1} + f a (L u^n + s^n),
//   f = 1 / (1 + t), g = (1 - t) f, t = (eta_x + eta_z) dt / 2, a = v^2 dt^2,
// with L the order-2R Laplacian (zero outside the padded grid, so L is
// symmetric), u^0 = u^{-1} = 0, residual e_n = R u^{n+1} - d_obs,n (R the
// bilinear receiver sampling) and phi = w/2 sum_n |e_n|^2 per shot of weight
// w.  Its exact discrete adjoint, for k = nt .. 1 with mu^{nt+1} = mu^{nt+2} = 0:
//   mu^k = w R^T e_{k-1} + 2 f mu^{k+1} + L (f a mu^{k+1}) - g mu^{k+2},
//   dphi/da = sum_{k=1..nt} mu^k f (L u^{k-1} + s^{k-1}).
// The forward pass keeps a whole history in HBM (no checkpointing: a shot
// of the 461 x 151 grid takes 0.78 GB).  Then dphi/da of the padded grid is
// folded back onto the physical nodes (the transpose of the edge extension
// into the damping pad) and chained to the velocity: dphi/dv = 2 v dt^2
// dphi/da.
//
// The forward pass normally runs on the on-chip (or L2) cluster modelling
// kernel, which streams out L u^n of every step, the only part of the
// forward field the adjoint pass needs (its gradient term then costs one
// pointwise read per point-step instead of a staged tile and a second
// Laplacian), and leaves its traces for adj_residual_kernel;
// adj_fwd_kernel is the per-step form for grids neither can hold (and order
// 16), which keeps its time levels in two adjoint slots and writes the
// same history.  The per-step kernels here run over all instances at once
// (blockIdx.y = instance), one launch per time step (the time loops replay as
// one CUDA graph).  They stage the fields their Laplacians read in
// shared-memory tiles and give each thread a few rows of one float4 group.
// The receiver transpose adds the four corner contributions in four ordered
// passes into one of two separate fields, one step ahead, which the adjoint
// step folds into mu.
#include <algorithm>

#include "internal.cuh"
#include "stencil.cuh"

namespace empso {

namespace {

struct SrcCorner {
    int I0, J0;
    float w[4];
};

__device__ __forceinline__ SrcCorner src_corner(float x, float z, const GridDev &g)
{
    SrcCorner c;
    const float fx = x / g.hx + (float)g.pad, fz = z / g.hz + (float)g.pad;
    c.I0 = min(max((int)floorf(fx), 0), g.NX - 2);
    c.J0 = min(max((int)floorf(fz), 0), g.NZ - 2);
    const float ax = fx - (float)c.I0, az = fz - (float)c.J0;
    c.w[0] = (1.f - ax) * (1.f - az);
    c.w[1] = ax * (1.f - az);
    c.w[2] = (1.f - ax) * az;
    c.w[3] = ax * az;
    return c;
}

// bilinear source weight of padded node (I, J)
__device__ __forceinline__ float src_weight(const SrcCorner &c, int I, int J)
{
    if (J == c.J0) return I == c.I0 ? c.w[0] : (I == c.I0 + 1 ? c.w[1] : 0.f);
    if (J == c.J0 + 1) return I == c.I0 ? c.w[2] : (I == c.I0 + 1 ? c.w[3] : 0.f);
    return 0.f;
}

// B = f a per model (m = blockIdx.y)
__global__ void adj_prep_kernel(GridDev g, const float *a, float *B)
{
    const long long off = (long long)blockIdx.y * g.field;
    const long long pts = (long long)g.NX * g.NZ;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < pts;
         e += (long long)gridDim.x * blockDim.x) {
        const int J = (int)(e / g.NX), I = (int)(e % g.NX);
        const long long k = (long long)(J + HALO) * g.pitch + I + HALO;
        const float t = g.ex[I + HALO] + g.ez[J + HALO];
        B[off + k] = a[off + k] / (1.f + t);
    }
}

// The per-point kernels work on tiles of TW float4 groups (4 TW points) by
// TT = 8 TZ rows; each of the block's TW x 8 threads computes TZ consecutive
// rows of one group.  The fields that enter a Laplacian are staged first,
// with R rows and XG = ceil(R / 4) groups of halo on every side, in shared
// memory.  The forward step takes TZ = 1 (its Laplacian reads one field; more
// rows per thread cost it registers and occupancy).  The adjoint step takes
// TZ = 4 when that still gives every SM enough blocks (less halo re-read, one
// wave), else 2 or 1 (more, smaller blocks to fill the GPU).
constexpr int TW = 16, TILE_THREADS = TW * 8;
constexpr int FWD_TZ8 = 4;   // forward rows per thread at radius 8 when the tiles fill the GPU

template <int R> struct Tile {
    static constexpr int XG = (R + 3) / 4;     // halo groups each side
    static constexpr int W = TW + 2 * XG;      // staged groups per row
};

__host__ __device__ inline int tiles_x(const GridDev &g) { return (g.NQ + TW - 1) / TW; }

// 16-byte asynchronous global -> shared copy; an invalid cell is filled with
// zeros and reads nothing (the source operand then only names the buffer)
__device__ __forceinline__ void cp_async16_zfill(void *sdst, const void *gsrc, bool valid)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(gsrc), "r"(valid ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// rows J0 - R .. J0 + TT - 1 + R, groups q0 - XG .. q0 + TW - 1 + XG of buffer
// U into S[TT + 2R][W] by asynchronous copies (complete after
// cp_async_wait_all and a barrier); cells outside the buffer read as zero
template <int R, int TT>
__device__ __forceinline__ void stage_tile(float4 *S, const float4 *__restrict__ U, int J0, int q0,
                                           const GridDev &g)
{
    constexpr int XG = Tile<R>::XG, W = Tile<R>::W, H = TT + 2 * R;
    const int p4 = g.pitch / 4;
    for (int c = threadIdx.x; c < W * H; c += TILE_THREADS) {
        const int row = J0 - R + c / W + HALO;      // buffer row
        const int grp = q0 - XG + HALO4 + c % W;    // buffer group of interior group q0 - XG + c % W
        const bool ok = row >= 0 && row < g.rows && grp >= 0 && grp < p4;
        cp_async16_zfill(S + c, ok ? U + (long long)row * p4 + grp : U, ok);
    }
}

// the same tile of the pointwise product of buffers X and Y (a fixed trip
// count, so that every thread's loads can be in flight together)
template <int R, int TT>
__device__ __forceinline__ void stage_tile_product(float4 *S, const float4 *__restrict__ X,
                                                   const float4 *__restrict__ Y, int J0, int q0,
                                                   const GridDev &g)
{
    constexpr int XG = Tile<R>::XG, W = Tile<R>::W, H = TT + 2 * R;
    constexpr int NIT = (W * H + TILE_THREADS - 1) / TILE_THREADS;
    const int p4 = g.pitch / 4;
#pragma unroll
    for (int it = 0; it < NIT; ++it) {
        const int c = threadIdx.x + it * TILE_THREADS;
        const int row = J0 - R + c / W + HALO;
        const int grp = q0 - XG + HALO4 + c % W;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (c < W * H && row >= 0 && row < g.rows && grp >= 0 && grp < p4) {
            const float4 x = X[(long long)row * p4 + grp], y = Y[(long long)row * p4 + grp];
            v = make_float4(x.x * y.x, x.y * y.y, x.z * y.z, x.w * y.w);
        }
        if (c < W * H) S[c] = v;
    }
}

// the staged x-line of the group at tile row sr, column sc (XG groups each side)
template <int R, int W = Tile<R>::W>
__device__ __forceinline__ void tile_xline(const float4 *S, int sr, int sc, float *xs)
{
    if (Tile<R>::XG == 1)
        xline1(S[sr * W + sc - 1], S[sr * W + sc], S[sr * W + sc + 1], xs);
    else
        xline2(S[sr * W + sc - 2], S[sr * W + sc - 1], S[sr * W + sc], S[sr * W + sc + 1], S[sr * W + sc + 2],
               xs);
}

// Laplacian of the four points of the staged group at tile row sr, column sc:
// z-neighbours as whole float4s, x-neighbours from the groups left and right
// (the modelling kernels' operator, stencil.cuh)
template <int R>
__device__ __forceinline__ float4 lap4_tile(const float4 *S, int sr, int sc, const GridDev &g)
{
    constexpr int W = Tile<R>::W;
    float4 w[2 * R + 1];
#pragma unroll
    for (int m = 0; m <= 2 * R; ++m) w[m] = S[(sr - R + m) * W + sc];
    float xs[4 * (2 * Tile<R>::XG + 1)];
    tile_xline<R>(S, sr, sc, xs);
    float2 l01, l23;
    lap_group<R>(w, xs, g.cxm, g.czm, g.cres, l01, l23);
    return make_float4(l01.x, l01.y, l23.x, l23.y);
}

// The same operator summed as written (centre weight c_0, pair sums): the
// adjoint step's form, where its FP32 rounding only enters the gradient and
// the differences would cost the step registers it does not have
template <int R, int W = Tile<R>::W>
__device__ __forceinline__ float4 lap4_tile_sum(const float4 *S, int sr, int sc, const GridDev &g)
{
    constexpr int XG = Tile<R>::XG, O = 4 * XG;
    float s[4 * (2 * XG + 1)];
    tile_xline<R, W>(S, sr, sc, s);
    float o[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) o[i] = g.cxm[0] * s[O + i];
#pragma unroll
    for (int m = 1; m <= R; ++m) {
        const float4 zm = S[(sr - m) * W + sc], zp = S[(sr + m) * W + sc];
        const float zs[4] = {zm.x + zp.x, zm.y + zp.y, zm.z + zp.z, zm.w + zp.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
            o[i] = fmaf(g.czm[m], zs[i], fmaf(g.cxm[m], s[O + i - m] + s[O + i + m], o[i]));
    }
    return make_float4(o[0], o[1], o[2], o[3]);
}

__device__ __forceinline__ float lane_of(const float4 &v, int i)
{
    return i == 0 ? v.x : (i == 1 ? v.y : (i == 2 ? v.z : v.w));
}

// Lanes past the last column (I >= NX) stay zero.

// One forward step n of every instance.  The time levels live in two of the
// instance's adjoint slots (free until the backward pass, L2-resident): u^n in
// slot n mod 2, and u^{n+1} overwrites u^{n-1} in the other one, point by
// point by the thread that read it.  The history slot n + 1 takes L u^n (the
// source term excluded): the pointwise history the adjoint step reads, as the
// cluster kernels' forward passes write it.
__device__ __forceinline__ float *fwd_level(const GridDev &g, const AdjInst &in, int n)
{
    return in.mu + (long long)(n % 2) * g.field;
}

template <int R, int TZ>
__global__ void __launch_bounds__(TILE_THREADS) adj_fwd_kernel(GridDev g, const AdjInst *__restrict__ insts, int n)
{
    constexpr int W = Tile<R>::W, XG = Tile<R>::XG, TT = 8 * TZ;
    __shared__ float4 S[(TT + 2 * R) * W];
    const AdjInst in = insts[blockIdx.y];
    // block 0 only records e_{n-1} = R u^n - d_obs,n-1 (u^n is complete),
    // beside the other blocks' stencil work
    if (blockIdx.x == 0) {
        if (n < 1) return;
        const float *uf = fwd_level(g, in, n);
        for (int r = threadIdx.x; r < in.nrec; r += blockDim.x) {
            const float2 p = in.rec[r];
            const SrcCorner c = src_corner(p.x, p.y, g);
            const long long kk = (long long)(c.J0 + HALO) * g.pitch + c.I0 + HALO;
            const float d = c.w[0] * uf[kk] + c.w[1] * uf[kk + 1] + c.w[2] * uf[kk + g.pitch] +
                            c.w[3] * uf[kk + g.pitch + 1];
            in.E[(long long)(n - 1) * in.nrec + r] = d - in.dobs[(long long)(n - 1) * in.nrec + r];
        }
        return;
    }
    const int t = blockIdx.x - 1, ntx = tiles_x(g);
    const int q0 = (t % ntx) * TW, J0 = (t / ntx) * TT;
    const int p4 = g.pitch / 4;
    // u^{n-1} (zero at n = 0) and u^{n+1} share a slot: no restrict, the
    // read of a point comes before its write in the same thread
    const float4 *u = reinterpret_cast<const float4 *>(fwd_level(g, in, n));
    const float4 *um = reinterpret_cast<const float4 *>(fwd_level(g, in, n + 1));
    float4 *u1 = reinterpret_cast<float4 *>(fwd_level(g, in, n + 1));
    float4 *hl = reinterpret_cast<float4 *>(in.H + (long long)(n + 1) * g.field);
    const float4 *a4 = reinterpret_cast<const float4 *>(in.a);
    stage_tile<R, TT>(S, u, J0, q0, g);
    cp_async_wait_all();
    __syncthreads();
    const int lx = threadIdx.x % TW, ly = threadIdx.x / TW, q = q0 + lx;
    if (q >= g.NQ) return;
    const SrcCorner sc = src_corner(in.sx, in.sz, g);
    const float rn = g.wavelet[n] / (g.hx * g.hz);
    const float4 ex = reinterpret_cast<const float4 *>(g.ex + HALO)[q];
#pragma unroll
    for (int r = 0; r < TZ; ++r) {
        const int J = J0 + ly * TZ + r;
        if (J >= g.NZ) break;
        const int sr = ly * TZ + r + R;
        const long long k4 = (long long)(J + HALO) * p4 + HALO4 + q;
        const float4 lap = lap4_tile<R>(S, sr, lx + XG, g);
        const float4 c = S[sr * W + lx + XG], m = um[k4], av = a4[k4];
        const float ez = g.ez[J + HALO];
        float o[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int I = 4 * q + i;
            const float t = lane_of(ex, i) + ez;
            const float li = fmaf(src_weight(sc, I, J), rn, lane_of(lap, i));
            o[i] = I < g.NX ? (2.f * lane_of(c, i) - (1.f - t) * lane_of(m, i) + lane_of(av, i) * li) / (1.f + t)
                            : 0.f;
        }
        u1[k4] = make_float4(o[0], o[1], o[2], o[3]);
        __stcs(hl + k4, lap);                // written once, read by the backward pass
    }
}

// Scatter of the receiver term J^kk = w R^T e_{kk-1} into J slot kk % 4 (zero
// before; the one-step kernel clears it again after reading, the two-step
// kernel's scatter zeroes it first): corner c of every receiver in pass c;
// receivers sharing a cell meet in an atomic add.  Run by one block.
__device__ __forceinline__ void scatter_receiver_term(const GridDev &g, const AdjInst &in, int kk)
{
    float *J = in.J + (long long)(kk % 4) * g.field;
    for (int c = 0; c < 4; ++c) {
        for (int r = threadIdx.x; r < in.nrec; r += blockDim.x) {
            const float2 p = in.rec[r];
            const SrcCorner sc = src_corner(p.x, p.y, g);
            const long long q = (long long)(sc.J0 + (c >> 1) + HALO) * g.pitch + sc.I0 + (c & 1) + HALO;
            atomicAdd(J + q, in.w * sc.w[c] * in.E[(long long)(kk - 1) * in.nrec + r]);
        }
        __syncthreads();
    }
}

// the receiver term of the first adjoint step (one block per instance)
__global__ void adj_scatter_kernel(GridDev g, const AdjInst *__restrict__ insts, int kk)
{
    scatter_receiver_term(g, insts[blockIdx.x], kk);
}

// the receiver terms of the first two adjoint steps kk and kk - 1 (the first
// two-step launch's)
__global__ void adj_scatter2_kernel(GridDev g, const AdjInst *__restrict__ insts, int kk)
{
    scatter_receiver_term(g, insts[blockIdx.x], kk);
    if (kk >= 2) scatter_receiver_term(g, insts[blockIdx.x], kk - 1);
}

// One adjoint step k, per point:
//   mu^k = 2 f mu^{k+1} + L Q^{k+1} - g mu^{k+2} + J^k   (J^k then cleared),
//   G += mu^k f (L u^{k-1} + s^{k-1}),
// with Q^{k+1} = f a mu^{k+1} formed as the tile is staged.  J is read only
// on the instance's receiver rows.  Block 0 meanwhile scatters J^{k-1} into
// the other J slot for the next step.  The history holds L u^{k-1} in slot k
// (every forward pass writes it), read per point past L2's keep-set.  mu
// rotates through `slots` slots: 4 beside the two-step kernel, else 2, where
// mu^k overwrites mu^{k+2} point by point in the thread that read it (the
// halo reads of neighbouring tiles are of mu^{k+1} only), which keeps the
// backward pass's fields within L2 for more instances.
template <int R, int TZ>
__global__ void __launch_bounds__(TILE_THREADS, 8) adj_step_kernel(GridDev g, const AdjInst *__restrict__ insts,
                                                                   int k, int slots)
{
    constexpr int W = Tile<R>::W, XG = Tile<R>::XG, TT = 8 * TZ;
    __shared__ float4 SQ[(TT + 2 * R) * W];
    const AdjInst in = insts[blockIdx.y];
    if (blockIdx.x == 0) {
        if (k >= 2) scatter_receiver_term(g, in, k - 1);
        return;
    }
    const int t = blockIdx.x - 1, ntx = tiles_x(g);
    const int q0 = (t % ntx) * TW, J0 = (t / ntx) * TT;
    const int p4 = g.pitch / 4;
    float4 *mk = reinterpret_cast<float4 *>(in.mu + (long long)(k % slots) * g.field);
    const float4 *m1 = reinterpret_cast<const float4 *>(in.mu + (long long)((k + 1) % slots) * g.field);
    const float4 *m2 = reinterpret_cast<const float4 *>(in.mu + (long long)((k + 2) % slots) * g.field);
    float4 *J4 = reinterpret_cast<float4 *>(in.J + (long long)(k % 4) * g.field);
    const float4 *u = reinterpret_cast<const float4 *>(in.H + (long long)k * g.field);   // L u^{k-1}
    const float4 *B4 = reinterpret_cast<const float4 *>(in.B);
    float4 *G4 = reinterpret_cast<float4 *>(in.G);
    stage_tile_product<R, TT>(SQ, B4, m1, J0, q0, g);
    cp_async_wait_all();
    __syncthreads();
    const int lx = threadIdx.x % TW, ly = threadIdx.x / TW, q = q0 + lx;
    if (q >= g.NQ) return;
    const SrcCorner sc = src_corner(in.sx, in.sz, g);
    const float rn = g.wavelet[k - 1] / (g.hx * g.hz);
    const float4 ex = reinterpret_cast<const float4 *>(g.ex + HALO)[q];
#pragma unroll
    for (int r = 0; r < TZ; ++r) {
        const int J = J0 + ly * TZ + r;
        if (J >= g.NZ) break;
        const int sr = ly * TZ + r + R;
        const long long k4 = (long long)(J + HALO) * p4 + HALO4 + q;
        const float4 lq = lap4_tile_sum<R>(SQ, sr, lx + XG, g);
        const float4 lu = __ldcs(u + k4);
        const float4 a1 = m1[k4], a2 = m2[k4];
        const bool jrow = J >= in.jr0 && J <= in.jr1;
        const float4 jj = jrow ? J4[k4] : make_float4(0.f, 0.f, 0.f, 0.f);
        if (jj.x != 0.f || jj.y != 0.f || jj.z != 0.f || jj.w != 0.f) J4[k4] = make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 gg = G4[k4];
        const float ez = g.ez[J + HALO];
        float mo[4], go[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int I = 4 * q + i;
            const float t = lane_of(ex, i) + ez;
            const float f = 1.f / (1.f + t);
            const float m = I < g.NX ? 2.f * f * lane_of(a1, i) + lane_of(lq, i) - (1.f - t) * f * lane_of(a2, i) +
                                           lane_of(jj, i)
                                     : 0.f;
            mo[i] = m;
            const float li = fmaf(src_weight(sc, I, J), rn, lane_of(lu, i));
            go[i] = fmaf(m / (1.f + t), li, lane_of(gg, i));
        }
        mk[k4] = make_float4(mo[0], mo[1], mo[2], mo[3]);
        G4[k4] = make_float4(go[0], go[1], go[2], go[3]);
    }
}

// Two adjoint steps per launch, k and k - 1, for the pointwise history (the
// cluster kernels' forward pass).  The block's tile T (rows J0 .. J0 + T2 - 1,
// groups q0 .. q0 + TW - 1) needs mu^k on T and on one stencil halo around it
// (region E) for the second step's L(f a mu^k), and mu^k on E needs
// f a mu^{k+1} on two halos (region E2).  So the block stages
// Q1 = f a mu^{k+1} on E2 (keeping mu^{k+1} on E), computes mu^k on E (the
// halo part again where the neighbouring tiles compute it too, in the same
// operation order, so with the same result), forms Q0 = f a mu^k on E in
// shared memory and computes mu^{k-1} on T.  The gradient takes both steps'
// terms on T, in the one-step order, with one read and one write of G.  mu
// lives in four rolling slots (k mod 4): a launch reads mu^{k+1}, mu^{k+2} and
// writes mu^k, mu^{k-1}, so a neighbour's halo reads never meet a slot being
// written.  J^k and J^{k-1} are only read here (a neighbour tile reads a
// cell's J in its halo); block 0 zeroes the next launch's two J slots on the
// receiver rows and scatters J^{k-2}, J^{k-3} into them.
constexpr int T2 = 32;            // rows of a two-step tile
constexpr int T2_THREADS = 256;

__device__ __forceinline__ void zero_receiver_rows(const GridDev &g, const AdjInst &in, int kk)
{
    float *J = in.J + (long long)(kk % 4) * g.field;
    const long long r0 = (long long)(max(in.jr0, -HALO) + HALO) * g.pitch;
    const long long n = (long long)(min(in.jr1, g.NZ + HALO - 1) - max(in.jr0, -HALO) + 1) * g.pitch;
    for (long long e = threadIdx.x; e < n; e += blockDim.x) J[r0 + e] = 0.f;
    __syncthreads();
}

template <int R>
__global__ void __launch_bounds__(T2_THREADS, 4) adj_step2_kernel(GridDev g, const AdjInst *__restrict__ insts,
                                                                  int k)
{
    constexpr int XG = Tile<R>::XG;
    constexpr int W1 = TW + 4 * XG, H1 = T2 + 4 * R;     // region E2
    constexpr int W0 = TW + 2 * XG, H0 = T2 + 2 * R;     // region E
    __shared__ float4 S1[H1 * W1], S0[H0 * W0], M1[H0 * W0], MK[T2 * TW];
    const AdjInst in = insts[blockIdx.y];
    if (blockIdx.x == 0) {
        for (int kk = k - 2; kk >= max(1, k - 3); --kk) {
            zero_receiver_rows(g, in, kk);
            scatter_receiver_term(g, in, kk);
        }
        return;
    }
    const int t = blockIdx.x - 1, ntx = tiles_x(g);
    const int q0 = (t % ntx) * TW, J0 = (t / ntx) * T2;
    const int p4 = g.pitch / 4;
    float4 *mu0 = reinterpret_cast<float4 *>(in.mu + (long long)(k % 4) * g.field);          // mu^k
    float4 *mu_1 = reinterpret_cast<float4 *>(in.mu + (long long)((k - 1) % 4) * g.field);   // mu^{k-1}
    const float4 *m1 = reinterpret_cast<const float4 *>(in.mu + (long long)((k + 1) % 4) * g.field);
    const float4 *m2 = reinterpret_cast<const float4 *>(in.mu + (long long)((k + 2) % 4) * g.field);
    const float4 *J0f = reinterpret_cast<const float4 *>(in.J + (long long)(k % 4) * g.field);
    const float4 *J1f = reinterpret_cast<const float4 *>(in.J + (long long)((k - 1) % 4) * g.field);
    const float4 *P0 = reinterpret_cast<const float4 *>(in.H + (long long)k * g.field);          // L u^{k-1}
    const float4 *P1 = reinterpret_cast<const float4 *>(in.H + (long long)(k - 1) * g.field);    // L u^{k-2}
    const float4 *B4 = reinterpret_cast<const float4 *>(in.B);
    float4 *G4 = reinterpret_cast<float4 *>(in.G);
    // Q1 = f a mu^{k+1} on E2 (zero outside the buffer), mu^{k+1} kept on E
    for (int c = threadIdx.x; c < H1 * W1; c += T2_THREADS) {
        const int tr = c / W1, tc = c % W1;
        const int row = J0 - 2 * R + tr + HALO, grp = q0 - 2 * XG + HALO4 + tc;   // buffer coordinates
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f), y = v;
        if (row >= 0 && row < g.rows && grp >= 0 && grp < p4) {
            const float4 x = B4[(long long)row * p4 + grp];
            y = m1[(long long)row * p4 + grp];
            v = make_float4(x.x * y.x, x.y * y.y, x.z * y.z, x.w * y.w);
        }
        S1[c] = v;
        if (tr >= R && tr < R + H0 && tc >= XG && tc < XG + W0) M1[(tr - R) * W0 + tc - XG] = y;
    }
    __syncthreads();
    const SrcCorner sc = src_corner(in.sx, in.sz, g);
    const float rn0 = g.wavelet[k - 1] / (g.hx * g.hz), rn1 = g.wavelet[k - 2] / (g.hx * g.hz);
    // step k on E; Q0 = f a mu^k on E
    for (int c = threadIdx.x; c < H0 * W0; c += T2_THREADS) {
        const int er = c / W0, ec = c % W0;
        const int J = J0 - R + er, q = q0 - XG + ec;
        float4 mk = make_float4(0.f, 0.f, 0.f, 0.f), bq = mk;
        if (J >= 0 && J < g.NZ && q >= 0 && q < g.NQ) {
            const long long k4 = (long long)(J + HALO) * p4 + HALO4 + q;
            const float4 lq = lap4_tile_sum<R, W1>(S1, er + R, ec + XG, g);
            const float4 a1 = M1[c], a2 = m2[k4];
            const bool jrow = J >= in.jr0 && J <= in.jr1;
            const float4 jj = jrow ? J0f[k4] : make_float4(0.f, 0.f, 0.f, 0.f);
            const float4 ex = reinterpret_cast<const float4 *>(g.ex + HALO)[q];
            const float ez = g.ez[J + HALO];
            float mo[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int I = 4 * q + i;
                const float tt = lane_of(ex, i) + ez;
                const float f = 1.f / (1.f + tt);
                mo[i] = I < g.NX ? 2.f * f * lane_of(a1, i) + lane_of(lq, i) - (1.f - tt) * f * lane_of(a2, i) +
                                       lane_of(jj, i)
                                 : 0.f;
            }
            mk = make_float4(mo[0], mo[1], mo[2], mo[3]);
            const float4 b = B4[k4];
            bq = make_float4(b.x * mk.x, b.y * mk.y, b.z * mk.z, b.w * mk.w);
            const int lr = J - J0, lx = q - q0;
            if (lr >= 0 && lr < T2 && lx >= 0 && lx < TW) {
                mu0[k4] = mk;
                MK[lr * TW + lx] = mk;
            }
        }
        S0[c] = bq;
    }
    __syncthreads();
    // step k - 1 on T, and both steps' gradient terms
    for (int c = threadIdx.x; c < T2 * TW; c += T2_THREADS) {
        const int lr = c / TW, lx = c % TW;
        const int J = J0 + lr, q = q0 + lx;
        if (J >= g.NZ || q >= g.NQ) continue;
        const long long k4 = (long long)(J + HALO) * p4 + HALO4 + q;
        const float4 lq = lap4_tile_sum<R, W0>(S0, lr + R, lx + XG, g);
        const float4 mk = MK[c], a1 = M1[(lr + R) * W0 + lx + XG];
        const bool jrow = J >= in.jr0 && J <= in.jr1;
        const float4 jj = jrow ? J1f[k4] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 gg = G4[k4], p0 = P0[k4], p1 = P1[k4];
        const float4 ex = reinterpret_cast<const float4 *>(g.ex + HALO)[q];
        const float ez = g.ez[J + HALO];
        float mo[4], go[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int I = 4 * q + i;
            const float tt = lane_of(ex, i) + ez;
            const float f = 1.f / (1.f + tt);
            const float m = I < g.NX ? 2.f * f * lane_of(mk, i) + lane_of(lq, i) - (1.f - tt) * f * lane_of(a1, i) +
                                           lane_of(jj, i)
                                     : 0.f;
            mo[i] = m;
            const float w = src_weight(sc, I, J);
            const float l0 = fmaf(w, rn0, lane_of(p0, i)), l1 = fmaf(w, rn1, lane_of(p1, i));
            go[i] = fmaf(m / (1.f + tt), l1, fmaf(lane_of(mk, i) / (1.f + tt), l0, lane_of(gg, i)));
        }
        mu_1[k4] = make_float4(mo[0], mo[1], mo[2], mo[3]);
        G4[k4] = make_float4(go[0], go[1], go[2], go[3]);
    }
}

// residual e_n = R u^{n+1} - d_obs,n (one block per instance), u^{n+1} in the
// rotating slots of the per-step forward pass
__global__ void adj_record_kernel(GridDev g, const AdjInst *__restrict__ insts, int n)
{
    const AdjInst in = insts[blockIdx.x];
    const float *u = fwd_level(g, in, n + 1);
    for (int r = threadIdx.x; r < in.nrec; r += blockDim.x) {
        const float2 p = in.rec[r];
        const SrcCorner c = src_corner(p.x, p.y, g);
        const long long k = (long long)(c.J0 + HALO) * g.pitch + c.I0 + HALO;
        const float d = c.w[0] * u[k] + c.w[1] * u[k + 1] + c.w[2] * u[k + g.pitch] +
                        c.w[3] * u[k + g.pitch + 1];
        in.E[(long long)n * in.nrec + r] = d - in.dobs[(long long)n * in.nrec + r];
    }
}

// e_n = d_n - d_obs,n of every instance in place, where the on-chip forward
// pass left its traces d_n = R u^{n+1} in E (blockIdx.y = instance)
__global__ void adj_residual_kernel(const AdjInst *__restrict__ insts, int nt)
{
    const AdjInst in = insts[blockIdx.y];
    const long long n = (long long)nt * in.nrec;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        in.E[i] -= in.dobs[i];
}

// phi of every instance: w/2 sum e^2 in a fixed order.  Pass 1: block b of
// instance q (blockIdx.y) sums chunk b of its residuals into part[q][b];
// pass 2 adds the MISFIT_PARTS partials in order.
constexpr int MISFIT_PARTS = 64;

__global__ void adj_misfit_part_kernel(const AdjInst *__restrict__ insts, int nt, double *part)
{
    const AdjInst in = insts[blockIdx.y];
    __shared__ double red[32];
    const long long n = (long long)nt * in.nrec;
    const long long chunk = (n + MISFIT_PARTS - 1) / MISFIT_PARTS;
    const long long i0 = blockIdx.x * chunk, i1 = i0 + chunk < n ? i0 + chunk : n;
    double s = 0.0;
    for (long long i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        const double e = in.E[i];
        s += e * e;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double v = 0.0;
        for (int w = 0; w < (int)blockDim.x / 32; ++w) v += red[w];
        part[(long long)blockIdx.y * MISFIT_PARTS + blockIdx.x] = v;
    }
}

__global__ void adj_misfit_sum_kernel(const AdjInst *__restrict__ insts, int n_inst, const double *part,
                                      double *phi)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n_inst) return;
    double v = 0.0;
    for (int b = 0; b < MISFIT_PARTS; ++b) v += part[(long long)q * MISFIT_PARTS + b];
    phi[q] = 0.5 * (double)insts[q].w * v;
}

// The fold of dphi/da from the padded grid onto the physical nodes is the
// transpose of the edge extension, separable in x and z: pass 1 sums, per
// padded row J and physical column i, every shot's G over the padded columns
// whose extension reads column i (one column inside, the pad and the edge
// column at either side) into T[m][J][i]; pass 2 sums T over the padded rows
// that read physical row j and chains to v: dphi/dv = 2 v dt^2 dphi/da.
__global__ void adj_fold_x_kernel(GridDev g, const AdjInst *__restrict__ insts, int S, float *T)
{
    const int m = blockIdx.y;
    const long long n = (long long)g.NZ * g.nx;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        const int J = (int)(e / g.nx), i = (int)(e % g.nx);
        const int I0 = i == 0 ? 0 : i + g.pad, I1 = i == g.nx - 1 ? g.NX - 1 : i + g.pad;
        float acc = 0.f;
        for (int s = 0; s < S; ++s) {
            const float *G = insts[m * S + s].G + (long long)(J + HALO) * g.pitch + HALO;
            for (int I = I0; I <= I1; ++I) acc += G[I];
        }
        T[(long long)m * n + e] = acc;
    }
}

// pass 2, and per model m the misfit = sum over shots (shot order)
__global__ void adj_fold_z_kernel(GridDev g, int S, const float *__restrict__ T,
                                  const float *__restrict__ vel, const double *phi, double *misfit,
                                  float *grad)
{
    const int m = blockIdx.y;
    const int np = g.nx * g.nz;
    if (blockIdx.x == 0 && threadIdx.x == 0 && misfit) {
        double v = 0.0;
        for (int s = 0; s < S; ++s) v += phi[m * S + s];
        misfit[m] = isfinite(v) ? v : __longlong_as_double(0x7ff0000000000000LL);
    }
    const float *Tm = T + (long long)m * g.NZ * g.nx;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < np; e += gridDim.x * blockDim.x) {
        const int j = e / g.nx, i = e % g.nx;
        const int J0 = j == 0 ? 0 : j + g.pad, J1 = j == g.nz - 1 ? g.NZ - 1 : j + g.pad;
        float acc = 0.f;
        for (int J = J0; J <= J1; ++J) acc += Tm[(long long)J * g.nx + i];
        const float v = vel[(long long)m * np + e];
        grad[(long long)m * np + e] = 2.f * v * g.dt * g.dt * acc;
    }
}

int grid_blocks(const GridDev &g)
{
    const long long items = (long long)g.NQ * g.NZ;
    long long b = (items + 255) / 256;
    return (int)(b > 4096 ? 4096 : b);
}

int tile_count(const GridDev &g, int TT) { return tiles_x(g) * ((g.NZ + TT - 1) / TT); }

using StepFn = void (*)(GridDev, const AdjInst *, int);
using Step1Fn = void (*)(GridDev, const AdjInst *, int, int);

StepFn fwd_fn(int R, int TZ)
{
    if (R == 8) return TZ == 4 ? adj_fwd_kernel<8, 4> : (TZ == 2 ? adj_fwd_kernel<8, 2> : adj_fwd_kernel<8, 1>);
    if (R == 4) return adj_fwd_kernel<4, 1>;
    return R == 2 ? adj_fwd_kernel<2, 1> : adj_fwd_kernel<1, 1>;
}
template <int TZ>
Step1Fn step_fn_z(int R)
{
    if (R == 8) return adj_step_kernel<8, TZ>;
    if (R == 4) return adj_step_kernel<4, TZ>;
    return R == 2 ? adj_step_kernel<2, TZ> : adj_step_kernel<1, TZ>;
}
Step1Fn step_fn(int R, int TZ) { return TZ == 4 ? step_fn_z<4>(R) : (TZ == 2 ? step_fn_z<2>(R) : step_fn_z<1>(R)); }

StepFn step2_fn(int R)
{
    if (R == 4) return adj_step2_kernel<4>;
    return R == 2 ? adj_step2_kernel<2> : adj_step2_kernel<1>;
}

// rows per thread of an adjoint-step launch over n_inst instances: 4 while
// that gives every SM 7 tile blocks (one wave at 8 resident), else 2 while
// that gives 3, else 1 (measured on the 461 x 151 grid: 16 shots run fastest
// at 4, 4 shots at 2)
int adj_rows_per_thread(const GridDev &g, int n_inst)
{
    int sms = 0, dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        sms = 1;
    if ((long long)tile_count(g, 32) * n_inst >= 7LL * sms) return 4;
    if ((long long)tile_count(g, 16) * n_inst >= 3LL * sms) return 2;
    return 1;
}

// rows per thread of the forward step: 1, except at radius 8, where a tile
// of 8 rows stages 3 times its rows (2R = 16 halo rows): there 4 rows (1.5
// times) while that gives every SM 7 tile blocks, else 2 while that gives 3
int adj_fwd_rows_per_thread(const GridDev &g, int n_inst)
{
    if (g.R < 8) return 1;
    int sms = 0, dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        sms = 1;
    if ((long long)tile_count(g, 32) * n_inst >= 7LL * sms) return FWD_TZ8;
    if ((long long)tile_count(g, 16) * n_inst >= 3LL * sms) return 2;
    return 1;
}

}  // namespace

cudaError_t launch_adj_prep(const GridDev &g, const float *a, float *B, int M, cudaStream_t st)
{
    adj_prep_kernel<<<dim3(grid_blocks(g), M), 256, 0, st>>>(g, a, B);
    return cudaGetLastError();
}

cudaError_t launch_adj_forward(const GridDev &g, const AdjInst *insts, int n_inst, int rec_threads,
                               cudaStream_t st)
{
    // step n also records e_{n-1} (in an extra block); the last record
    // follows the loop
    const int tz = adj_fwd_rows_per_thread(g, n_inst);
    const dim3 grid(tile_count(g, 8 * tz) + 1, n_inst);
    const StepFn fn = fwd_fn(g.R, tz);
    for (int n = 0; n < g.nt; ++n) fn<<<grid, TILE_THREADS, 0, st>>>(g, insts, n);
    adj_record_kernel<<<n_inst, rec_threads, 0, st>>>(g, insts, g.nt - 1);
    return cudaGetLastError();
}

cudaError_t launch_adj_residual(const GridDev &g, const AdjInst *insts, int n_inst, int rec_max,
                                cudaStream_t st)
{
    const long long n = (long long)g.nt * rec_max;
    adj_residual_kernel<<<dim3((unsigned)std::min<long long>((n + 255) / 256, 64), n_inst), 256, 0, st>>>(insts, g.nt);
    return cudaGetLastError();
}

cudaError_t launch_adj_backward(const GridDev &g, const AdjInst *insts, int n_inst, int n_all, int rec_threads,
                                cudaStream_t st)
{
    const int tz = adj_rows_per_thread(g, n_all);
    const Step1Fn fn = step_fn(g.R, tz);
    // two steps per launch while its tiles (4 resident per SM: 46.6 KB of
    // shared memory each) make at most two waves over all chains; beyond, the
    // one-step kernel's 8 blocks per SM hide more latency (461 x 151 grid:
    // 16 shots 28.4 -> 24.7 ms with two steps, 32 shots 43.8 -> 49.1)
    int sms = 0, dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        sms = 1;
    const long long tiles2 = (long long)tiles_x(g) * ((g.NZ + T2 - 1) / T2);
    if (g.R <= 4 && tiles2 * n_all <= 2LL * 4 * sms) {
        // the receiver terms of steps nt and nt - 1 first, each launch's
        // block 0 then scatters the next launch's two; an odd last step takes
        // the one-step kernel
        const dim3 grid2(tiles_x(g) * ((g.NZ + T2 - 1) / T2) + 1, n_inst);
        const StepFn fn2 = step2_fn(g.R);
        adj_scatter2_kernel<<<n_inst, rec_threads, 0, st>>>(g, insts, g.nt);
        int k = g.nt;
        for (; k >= 2; k -= 2) fn2<<<grid2, T2_THREADS, 0, st>>>(g, insts, k);
        if (k == 1) fn<<<dim3(tile_count(g, 8 * tz) + 1, n_inst), TILE_THREADS, 0, st>>>(g, insts, 1, 4);
        return cudaGetLastError();
    }
    // the receiver term of step nt first; each step's extra block then
    // scatters the next step's.  The rows per thread follow the instances of
    // all chains that run at once (n_all).
    const dim3 grid(tile_count(g, 8 * tz) + 1, n_inst);
    adj_scatter_kernel<<<n_inst, rec_threads, 0, st>>>(g, insts, g.nt);
    for (int k = g.nt; k >= 1; --k) fn<<<grid, TILE_THREADS, 0, st>>>(g, insts, k, 2);
    return cudaGetLastError();
}

// misfit[m] = sum over shots of phi (shot order), +inf when not finite
__global__ void adj_model_misfit_kernel(int M, int S, const double *phi, double *misfit)
{
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    double v = 0.0;
    for (int s = 0; s < S; ++s) v += phi[m * S + s];
    misfit[m] = isfinite(v) ? v : __longlong_as_double(0x7ff0000000000000LL);
}

cudaError_t launch_adj_misfit(const GridDev &g, const AdjInst *insts, int M, int S, double *phi,
                              double *misfit, double *part, cudaStream_t st)
{
    adj_misfit_part_kernel<<<dim3(MISFIT_PARTS, M * S), 256, 0, st>>>(insts, g.nt, part);
    adj_misfit_sum_kernel<<<(M * S + 127) / 128, 128, 0, st>>>(insts, M * S, part, phi);
    adj_model_misfit_kernel<<<(M + 127) / 128, 128, 0, st>>>(M, S, phi, misfit);
    return cudaGetLastError();
}

cudaError_t launch_adj_finish(const GridDev &g, const AdjInst *insts, int M, int S, const float *vel,
                              double *phi, double *misfit, float *grad, float *T, cudaStream_t st)
{
    // the misfit partials borrow the fold's scratch, which pass 1 of the fold
    // overwrites only after they are summed
    double *part = reinterpret_cast<double *>(T);
    adj_misfit_part_kernel<<<dim3(MISFIT_PARTS, M * S), 256, 0, st>>>(insts, g.nt, part);
    adj_misfit_sum_kernel<<<(M * S + 127) / 128, 128, 0, st>>>(insts, M * S, part, phi);
    const long long nT = (long long)g.NZ * g.nx;
    adj_fold_x_kernel<<<dim3((unsigned)((nT + 255) / 256), M), 256, 0, st>>>(g, insts, S, T);
    const int np = g.nx * g.nz;
    adj_fold_z_kernel<<<dim3((np + 255) / 256, M), 256, 0, st>>>(g, S, T, vel, phi, misfit, grad);
    return cudaGetLastError();
}

}  // namespace empso

// ---------------------------------------------------------------------------
// vector kernels of the local FWI driver (one model field [nz][nx])
// ---------------------------------------------------------------------------
namespace empso {

namespace {

// out = clip(v - alpha g, vmin, vmax)
__global__ void fwi_step_kernel(const float *v, const float *g, float alpha, float vmin, float vmax,
                                float *out, int n)
{
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x)
        out[e] = fminf(fmaxf(v[e] - alpha * g[e], vmin), vmax);
}

// r[0] = sum (a - b) c, r[1] = sum (a - b)^2, r[2] = sum (a - b)(c - d),
// r[3] = max |c|, r[4] = sum a; one block, fixed reduction order
__global__ void fwi_dots_kernel(const float *a, const float *b, const float *c, const float *d, int n,
                                double *r)
{
    __shared__ double red[5][32];
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, mx = 0.0, sa = 0.0;
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
        const double ab = b ? (double)a[e] - (double)b[e] : (double)a[e];
        const double cc = c[e];
        const double cd = d ? cc - (double)d[e] : cc;
        s0 += ab * cc;
        s1 += ab * ab;
        s2 += ab * cd;
        mx = fmax(mx, fabs(cc));
        sa += a[e];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s0 += __shfl_down_sync(0xffffffffu, s0, o);
        s1 += __shfl_down_sync(0xffffffffu, s1, o);
        s2 += __shfl_down_sync(0xffffffffu, s2, o);
        mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
        sa += __shfl_down_sync(0xffffffffu, sa, o);
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        red[0][w] = s0;
        red[1][w] = s1;
        red[2][w] = s2;
        red[3][w] = mx;
        red[4][w] = sa;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
        for (int i = 0; i < (int)blockDim.x / 32; ++i) {
            t[0] += red[0][i];
            t[1] += red[1][i];
            t[2] += red[2][i];
            t[3] = fmax(t[3], red[3][i]);
            t[4] += red[4][i];
        }
        for (int i = 0; i < 5; ++i) r[i] = t[i];
    }
}

}  // namespace

cudaError_t launch_fwi_step(const float *v, const float *g, float alpha, float vmin, float vmax,
                            float *out, int n, cudaStream_t st)
{
    fwi_step_kernel<<<(n + 255) / 256 > 1024 ? 1024 : (n + 255) / 256, 256, 0, st>>>(v, g, alpha, vmin,
                                                                                    vmax, out, n);
    return cudaGetLastError();
}

cudaError_t launch_fwi_dots(const float *a, const float *b, const float *c, const float *d, int n,
                            double *r, cudaStream_t st)
{
    fwi_dots_kernel<<<1, 1024, 0, st>>>(a, b, c, d, n, r);
    return cudaGetLastError();
}

}  // namespace empso
