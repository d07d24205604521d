// On-chip ("resident") variant of the persistent modelling launch: the same
// scheme and fused source/receiver/misfit work as wave.cu (section "Testing
// approach": 2nd order in time, 4th/8th order in space, damping layer, Ricker
// source, l2 misfit), but an instance's two time levels never leave the SMs.
//
// A thread-block cluster of C CTAs owns one instance at a time (taken from a
// global queue by cluster rank 0).  The padded grid is split by rows: CTA c
// holds rows [c*rows_c, (c+1)*rows_c) of u^n and u^{n-1}/u^{n+1} in its shared
// memory with R halo rows above and below, and keeps its share of the model
// field a = v^2 dt^2 in registers.  Every step each thread updates ROWS rows
// of one float4 column group (z-stencil from a register window, x-stencil from
// the neighbouring float4s in shared memory), writes u^{n+1} in place of
// u^{n-1}, and stores its slab's first/last R rows straight into the halo rows
// of the neighbouring CTAs (distributed shared memory).  One cluster barrier
// (release/acquire) per step orders it all.  Global memory is touched only for
// the model field (once per instance), the observed traces and the output.
#include <cooperative_groups.h>

#include "internal.cuh"
#include "stencil.cuh"

namespace cg = cooperative_groups;

namespace empso {

namespace {

constexpr int ROWS = 8;

__device__ __forceinline__ void set_comp(float4 &v, int l, float x)
{
    if (l == 0) v.x = x;
    else if (l == 1) v.y = x;
    else if (l == 2) v.z = x;
    else v.w = x;
}

// 4-byte asynchronous global -> shared copies (cp.async), grouped per step
__device__ __forceinline__ void cp_async4(void *smem_dst, const void *gsrc)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Double-buffered shared-memory staging of the wavelet sample and observed
// record each step needs: step n copies what step n + 1 uses and waits for
// those copies before its closing barrier, so no copy is in flight across a
// barrier (a release barrier would wait for it) and the copy latency hides
// under the stencil work.
constexpr int DEPTH = 2;

// Bilinear corners of (x, z) metres on the padded grid (lower corner clamped
// to NX-2 / NZ-2), as global padded indices.
__device__ __forceinline__ void corners(float x, float z, const GridDev &g, int &i0, int &j0,
                                        float w[4])
{
    const float fx = x / g.hx + (float)g.pad;
    const float fz = z / g.hz + (float)g.pad;
    i0 = min(max((int)floorf(fx), 0), g.NX - 2);
    j0 = min(max((int)floorf(fz), 0), g.NZ - 2);
    const float ax = fx - (float)i0, az = fz - (float)j0;
    w[0] = (1.f - ax) * (1.f - az);
    w[1] = ax * (1.f - az);
    w[2] = (1.f - ax) * az;
    w[3] = ax * az;
}

// C CTAs (ranks base .. base + C - 1 of the cluster; crank is the rank among
// them) run instance `in`; with HIST every u^{n+1} also goes to in.hist
template <int R, bool HIST>
__device__ void resident_instance(const GridDev &gs, const Inst &in, float4 *A4, float4 *B4,
                                  float4 *M4, float *ezs, float *wring, float *dring, float4 *rec_w,
                                  int *rec_k, int ring_pitch,
                                  int C, int crank, int base, cg::cluster_group &cluster, double *cred,
                                  double *wred, double *partial)
{
    const int tid = threadIdx.x;
    const int nth = blockDim.x;
    // scalars of the grid in registers (the descriptor lives in shared memory)
    const int NQ = gs.NQ, NZ = gs.NZ, NX = gs.NX, nt = gs.nt, pitch = gs.pitch;
    const float *__restrict__ gex = gs.ex;
    const float *__restrict__ gez = gs.ez;
    const float *__restrict__ gwav = gs.wavelet;
    const int sp4 = NQ + 2;                      // float4 per shared row (1 zero group each side)
    const int rows_c = (NZ + C - 1) / C;
    const int srows = rows_c + 2 * R;
    const int z0 = crank * rows_c;
    const int my_rows = max(0, min(NZ, z0 + rows_c) - z0);

    // zero both time levels (halos included) and load this slab of the model field
    for (int e = tid; e < 2 * srows * sp4; e += nth) A4[e] = make_float4(0.f, 0.f, 0.f, 0.f);
    // model slab pre-scaled by f = 1 / (1 + t), t = (eta_x + eta_z) dt / 2, so
    // that the damped update needs no division per point (see below)
    for (int e = tid; e < my_rows * NQ; e += nth) {
        const int r = e / NQ, qq = e % NQ;
        const float4 av =
            __ldg(reinterpret_cast<const float4 *>(in.a + (size_t)(z0 + r + HALO) * pitch + HALO) + qq);
        const float4 exq = __ldg(reinterpret_cast<const float4 *>(gex + HALO) + qq);
        const float ez = __ldg(gez + z0 + r + HALO);
        M4[r * NQ + qq] = make_float4(av.x / (1.f + (exq.x + ez)), av.y / (1.f + (exq.y + ez)),
                                      av.z / (1.f + (exq.z + ez)), av.w / (1.f + (exq.w + ez)));
    }
    for (int r = tid; r < my_rows; r += nth) ezs[r] = __ldg(gez + z0 + r + HALO);

    // work item: column group q and ROWS consecutive slab rows from r0.  Every
    // item computes exactly ROWS rows (no per-row conditions): the last item of
    // a column starts at my_rows - ROWS, overlapping its predecessor, and stores
    // only rows >= seg * ROWS.  rows_c >= ROWS keeps every read inside the slab
    // buffers even on a short last CTA.
    const int nseg = (my_rows + ROWS - 1) / ROWS;
    const bool active = tid < NQ * nseg;
    const int q = active ? tid % NQ : 0;
    const int seg = active ? tid / NQ : 0;
    const int r0 = active ? max(0, min(seg * ROWS, my_rows - ROWS)) : 0;
    const int kfirst = seg * ROWS - r0;          // first row this item stores
    const int klast = my_rows - r0;              // one past the last row it stores
    const int rc = ROWS;

    float4 ex = make_float4(0.f, 0.f, 0.f, 0.f);
    if (active) ex = __ldg(reinterpret_cast<const float4 *>(gex + HALO) + q);
    // update weight g = 2 / (1 + t) of rows without z-damping: per lane,
    // constant over the instance (g = 2 in the interior)
    const float2 gx01 = make_float2(2.f / (1.f + ex.x), 2.f / (1.f + ex.y));
    const float2 gx23 = make_float2(2.f / (1.f + ex.z), 2.f / (1.f + ex.w));
    float cx[R + 1], cz[R + 1];
#pragma unroll
    for (int m = 0; m <= R; ++m) {
        cx[m] = gs.cxm[m];
        cz[m] = gs.czm[m];
    }
    const float cres = gs.cres;

    // source: weights b / (hx hz) of the (up to) two rows and four lanes of
    // this item that hold one of its bilinear corners
    int s_i0, s_j0;
    float sw[4];
    corners(in.sx, in.sz, gs, s_i0, s_j0, sw);
    const float inv_cell = 1.f / (gs.hx * gs.hz);
    const int ks = s_j0 - (z0 + r0);             // item row of the upper corner row
    float4 sb0 = make_float4(0.f, 0.f, 0.f, 0.f), sb1 = sb0;
    bool src_here = false;
    if (active && s_i0 >= 4 * q - 1 && s_i0 <= 4 * q + 3 && ks + 1 >= 0 && ks < rc) {
        src_here = true;
#pragma unroll
        for (int l = 0; l < 4; ++l) {
            const int I = 4 * q + l;
            const float bx0 = (I == s_i0 ? 1.f : 0.f), bx1 = (I == s_i0 + 1 ? 1.f : 0.f);
            set_comp(sb0, l, (bx0 * sw[0] + bx1 * sw[1]) * inv_cell);
            set_comp(sb1, l, (bx0 * sw[2] + bx1 * sw[3]) * inv_cell);
        }
    }

    // receivers: bilinear corners and weights of every receiver, computed once
    // per instance; rec_k = float index of the lower-left corner in this CTA's
    // slab, or -1 when another CTA holds the receiver's lower corner row
    const int nrec = in.nrec;
    const float *__restrict__ dobs = in.dobs;
    for (int r = tid; r < nrec; r += nth) {
        const float2 pr = in.rec[r];
        int i0, j0;
        float w4[4];
        corners(pr.x, pr.y, gs, i0, j0, w4);
        const bool mine = j0 >= z0 && j0 < z0 + my_rows;
        rec_k[r] = mine ? (j0 - z0 + R) * (4 * sp4) + 4 + i0 : -1;
        rec_w[r] = make_float4(w4[0], w4[1], w4[2], w4[3]);
    }
    // staging prologue: the wavelet sample of step 0
    if (tid == 0 && nt > 0) cp_async4(wring, gwav);
    cp_async_commit();
    cp_async_wait<0>();
    float accf = 0.f;
    double acc = 0.0;
    (void)NX;
    (void)ring_pitch;

    cluster.sync();                                      // zeroed everywhere before halo stores

    // neighbours' views of both time-level buffers
    float4 *prev_A = nullptr, *prev_B = nullptr, *next_A = nullptr, *next_B = nullptr;
    if (crank > 0) {
        prev_A = cluster.map_shared_rank(A4, base + crank - 1);
        prev_B = cluster.map_shared_rank(B4, base + crank - 1);
    }
    if (crank < C - 1) {
        next_A = cluster.map_shared_rank(A4, base + crank + 1);
        next_B = cluster.map_shared_rank(B4, base + crank + 1);
    }
    const bool top_item = r0 < R;                        // may hold halo rows of the CTA above
    const bool bot_item = r0 + ROWS > rows_c - R;        // ... of the CTA below

    // history: this item's first row in slot n + 1 (advanced one field per step)
    float4 *hrow = nullptr;
    if (HIST && active)
        hrow = reinterpret_cast<float4 *>(in.hist) + (size_t)(z0 + r0 + HALO) * (pitch / 4) + 1 + q;
    float4 *cur = A4, *nxt = B4;
    for (int n = 0; n <= nt; ++n) {
        if (HIST) hrow += gs.field / 4;
        // stage wavelet sample n + 1 and record n (sampled in step n + 1); their
        // slots were last read in step n - 1, which the previous barrier closed
        {
            const int iw = n + 1, ir = n;
            if (tid == 0 && iw < nt) cp_async4(wring + iw % DEPTH, gwav + iw);
            if (dobs && ir < nt)
                for (int r = tid; r < nrec; r += nth)
                    if (rec_k[r] >= 0)
                        cp_async4(dring + (ir % DEPTH) * nrec + r, dobs + (size_t)ir * nrec + r);
            cp_async_commit();
        }
        if (n < nt && active) {
            const float rn = wring[n % DEPTH];
            const bool even = (n & 1) == 0;           // nxt is B4 on even steps, A4 on odd
            float4 *prevA = even ? prev_B : prev_A;
            float4 *nextA = even ? next_B : next_A;
            float4 w[2 * R + 1];
#pragma unroll
            for (int m = 0; m < 2 * R; ++m) w[m] = cur[(r0 + m) * sp4 + 1 + q];
#pragma unroll
            for (int k = 0; k < ROWS; ++k) {
                {
                    const int lr = R + r0 + k;           // shared row of the output
                    w[2 * R] = cur[(lr + R) * sp4 + 1 + q];
                    const float4 lft = cur[lr * sp4 + q];
                    const float4 rgt = cur[lr * sp4 + 2 + q];
                    const float4 um = nxt[lr * sp4 + 1 + q];
                    const float4 av = M4[(r0 + k) * NQ + q];
                    // Laplacian of lanes (0,1) and (2,3) with packed FP32x2 arithmetic;
                    // x and z parts accumulate separately (two independent chains)
                    const float2 c01 = lo2(w[R]), c23 = hi2(w[R]);
                    float xs[12];
                    xline1(lft, w[R], rgt, xs);
                    float2 lap01, lap23;
                    lap_group<R>(w, xs, cx, cz, cres, lap01, lap23);
                    if (src_here && (k == ks || k == ks + 1)) {
                        const float4 sb = (k == ks) ? sb0 : sb1;
                        lap01 = __ffma2_rn(make_float2(sb.x, sb.y), make_float2(rn, rn), lap01);
                        lap23 = __ffma2_rn(make_float2(sb.z, sb.w), make_float2(rn, rn), lap23);
                    }
                    // u^{n+1} = [2 u^n - (1 - t) u^{n-1} + a lap] / (1 + t)
                    //         = g (u^n - u^{n-1}) + u^{n-1} + (a f) lap,  g = 2 f, f = 1 / (1 + t)
                    // (a f is the pre-scaled model slab); one branch-free form for
                    // interior and damping layer, g per lane and row
                    const float ezk = ezs[r0 + k];
                    float2 g01 = gx01, g23 = gx23;
                    if (ezk != 0.f) {
                        g01 = make_float2(__fdividef(2.f, 1.f + (ex.x + ezk)), __fdividef(2.f, 1.f + (ex.y + ezk)));
                        g23 = make_float2(__fdividef(2.f, 1.f + (ex.z + ezk)), __fdividef(2.f, 1.f + (ex.w + ezk)));
                    }
                    const float2 um01 = make_float2(um.x, um.y), um23 = make_float2(um.z, um.w);
                    const float2 o01 = __ffma2_rn(g01, __fadd2_rn(c01, make_float2(-um.x, -um.y)),
                                                  __ffma2_rn(make_float2(av.x, av.y), lap01, um01));
                    const float2 o23 = __ffma2_rn(g23, __fadd2_rn(c23, make_float2(-um.z, -um.w)),
                                                  __ffma2_rn(make_float2(av.z, av.w), lap23, um23));
                    const float4 out = make_float4(o01.x, o01.y, o23.x, o23.y);
                    if (k >= kfirst && k < klast) {
                        nxt[lr * sp4 + 1 + q] = out;
                        if (HIST) __stcs(hrow + k * (pitch / 4), out);   // written once: evict first
                        // halo rows of the neighbours
                        const int rr = r0 + k;
                        if (top_item && prevA && rr < R) prevA[(rr + rows_c + R) * sp4 + 1 + q] = out;
                        if (bot_item && nextA && rr >= rows_c - R)
                            nextA[(rr - rows_c + R) * sp4 + 1 + q] = out;
                    }
                }
#pragma unroll
                for (int m = 0; m < 2 * R; ++m) w[m] = w[m + 1];
            }
        }
        // receivers sample u^n (record n - 1)
        if (n >= 1) {
            const float *cf = reinterpret_cast<const float *>(cur);
            const int sp = 4 * sp4;
            for (int r = tid; r < nrec; r += nth) {
                const int k0 = rec_k[r];
                if (k0 < 0) continue;
                const float4 w4 = rec_w[r];
                const float d = w4.x * cf[k0] + w4.y * cf[k0 + 1] + w4.z * cf[k0 + sp] +
                                w4.w * cf[k0 + sp + 1];
                if (in.traces) in.traces[(size_t)(n - 1) * nrec + r] = d;
                if (dobs) {
                    const float e = d - dring[((n - 1) % DEPTH) * nrec + r];
                    accf = fmaf(e, e, accf);
                }
            }
            if ((n & 31) == 0) {        // keep the FP32 partial short, carry in FP64
                acc += (double)accf;
                accf = 0.f;
            }
        }
        // this step's copies have landed; the barrier publishes them
        cp_async_wait<0>();
        cluster.sync();
        float4 *t = cur;
        cur = nxt;
        nxt = t;
    }
    cp_async_wait<0>();
    if (!dobs) accf = 0.f, acc = 0.0;
    acc += (double)accf;
    // fixed-order reduction: warps -> CTA -> cluster rank 0 (ranks in order)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((tid & 31) == 0) wred[tid >> 5] = acc;
    __syncthreads();
    if (tid < 32) {
        double v = (tid < nth / 32) ? wred[tid] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (tid == 0) *cluster.map_shared_rank(cred + crank, base) = v;
    }
    cluster.sync();
    if (crank == 0 && tid == 0) {
        double sum = 0.0;
        for (int c = 0; c < C; ++c) sum += cred[c];
        partial[in.out] = 0.5 * sum;
    }
}

// Work unit u of the queue: units[u] = {a, b, halves}.  halves = 0: the whole
// cluster runs instance a; halves = 1: ranks 0 .. C/2 - 1 run instance a and
// ranks C/2 .. C - 1 instance b, both of the same grid (so both halves pass
// the same number of cluster barriers).  Launches with no halved unit use the
// PAIRS = false instantiation, where the whole-cluster layout is constant.
// HIST (never with PAIRS) also writes the wavefield history.
template <int R, int NT, bool PAIRS, bool HIST>
__global__ void __launch_bounds__(NT, 1)
wave_resident_kernel(const GridDev *__restrict__ grids, const Inst *__restrict__ insts,
                     const int4 *__restrict__ units, int n_units, int *counter, int ring_pitch,
                     double *partial)
{
    extern __shared__ float4 smem4[];
    __shared__ int s_q;
    __shared__ double cred[16];
    __shared__ double wred[NT / 32];
    __shared__ GridDev sg;
    cg::cluster_group cluster = cg::this_cluster();
    const int C = (int)cluster.num_blocks();
    const int crank = (int)cluster.block_rank();
    for (;;) {
        if (crank == 0 && threadIdx.x == 0) {
            const int q = atomicAdd(counter, 1);
            for (int c = 0; c < C; ++c) *cluster.map_shared_rank(&s_q, c) = q;
        }
        cluster.sync();
        const int u = s_q;
        if (u >= n_units) break;
        const int4 un = units[u];
        const bool halves = PAIRS && un.z != 0;
        const int Ce = halves ? C / 2 : C;
        const int sub = halves ? (crank >= C / 2 ? 1 : 0) : 0;
        const int ce = crank - sub * Ce;
        const Inst in = insts[sub ? un.y : un.x];
        if (threadIdx.x == 0) sg = grids[in.grid];
        __syncthreads();
        const int rows_c = (sg.NZ + Ce - 1) / Ce;
        float4 *A4 = smem4;
        float4 *B4 = A4 + (size_t)(rows_c + 2 * R) * (sg.NQ + 2);
        float4 *M4 = B4 + (size_t)(rows_c + 2 * R) * (sg.NQ + 2);
        float *ezs = reinterpret_cast<float *>(M4 + (size_t)rows_c * sg.NQ);
        float *wring = ezs + (rows_c + 3) / 4 * 4;
        float *dring = wring + 4 * ((DEPTH + 3) / 4);
        float4 *rec_w = reinterpret_cast<float4 *>(dring + (DEPTH * ring_pitch + 3) / 4 * 4);
        int *rec_k = reinterpret_cast<int *>(rec_w + ring_pitch);
        resident_instance<R, HIST>(sg, in, A4, B4, M4, ezs, wring, dring, rec_w, rec_k, ring_pitch, Ce,
                             ce, sub * Ce, cluster, cred, wred, partial);
    }
}

constexpr int RES_NT = 512;

}  // namespace

int resident_max_threads() { return RES_NT; }
int resident_rows_per_thread() { return ROWS; }

// two time levels with halo rows, the slab of the model field, its damping
// rows, the staging buffers (wavelet samples, observed records) and the
// receiver tables, for shots of up to ring_pitch receivers
size_t resident_smem_bytes(const GridDev &g, int C, int ring_pitch)
{
    const int rows_c = (g.NZ + C - 1) / C;
    return sizeof(float4) * (2 * (size_t)(rows_c + 2 * g.R) * (g.NQ + 2) + (size_t)rows_c * g.NQ) +
           sizeof(float) * ((rows_c + 3) / 4 * 4 + 4 * ((DEPTH + 3) / 4) +
                            ((size_t)DEPTH * ring_pitch + 3) / 4 * 4) +
           (sizeof(float4) + sizeof(int)) * (size_t)ring_pitch;
}

// Does grid g run on a cluster of C CTAs?  Each CTA needs at least R rows (so
// halos come from the nearest neighbour only), no CTA may be empty, the work
// items must fit one thread each, and the two time levels plus the model slab
// the shared memory.
bool resident_fits(const GridDev &g, int C, int ring_pitch, size_t smem_limit)
{
    const int rows_c = (g.NZ + C - 1) / C;
    if (rows_c < g.R || rows_c < ROWS) return false;
    if ((C - 1) * rows_c >= g.NZ) return false;
    const int nseg = (rows_c + ROWS - 1) / ROWS;
    if (g.NQ * nseg > RES_NT) return false;
    return resident_smem_bytes(g, C, ring_pitch) <= smem_limit;
}

namespace {
template <int R, bool PAIRS, bool HIST>
cudaError_t configure_rp(size_t smem_bytes, int C)
{
    cudaError_t e = cudaFuncSetAttribute(wave_resident_kernel<R, RES_NT, PAIRS, HIST>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem_bytes);
    if (e != cudaSuccess) return e;
    if (C > 8)
        e = cudaFuncSetAttribute(wave_resident_kernel<R, RES_NT, PAIRS, HIST>,
                                 cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    return e;
}

template <int R>
cudaError_t configure_r(size_t smem_bytes, int C)
{
    cudaError_t e = configure_rp<R, false, false>(smem_bytes, C);
    if (e == cudaSuccess) e = configure_rp<R, true, false>(smem_bytes, C);
    return e != cudaSuccess ? e : configure_rp<R, false, true>(smem_bytes, C);
}

using ResidentFn = void (*)(const GridDev *, const Inst *, const int4 *, int, int *, int, double *);

ResidentFn resident_fn(int R, bool pairs, bool hist = false)
{
    if (hist) {
        if (R == 4) return wave_resident_kernel<4, RES_NT, false, true>;
        if (R == 2) return wave_resident_kernel<2, RES_NT, false, true>;
        return wave_resident_kernel<1, RES_NT, false, true>;
    }
    if (pairs) {
        if (R == 4) return wave_resident_kernel<4, RES_NT, true, false>;
        if (R == 2) return wave_resident_kernel<2, RES_NT, true, false>;
        return wave_resident_kernel<1, RES_NT, true, false>;
    }
    if (R == 4) return wave_resident_kernel<4, RES_NT, false, false>;
    if (R == 2) return wave_resident_kernel<2, RES_NT, false, false>;
    return wave_resident_kernel<1, RES_NT, false, false>;
}
}  // namespace

cudaError_t resident_configure(int R, size_t smem_bytes, int C)
{
    if (R == 4) return configure_r<4>(smem_bytes, C);
    if (R == 2) return configure_r<2>(smem_bytes, C);
    return configure_r<1>(smem_bytes, C);
}

int resident_max_clusters(int R, int C, int threads, size_t smem_bytes)
{
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(C * 64, 1, 1);
    cfg.blockDim = dim3(threads, 1, 1);
    cfg.dynamicSmemBytes = smem_bytes;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, resident_fn(R, false), &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

cudaError_t launch_wave_resident(int R, const GridDev *grids_dev, const Inst *insts, const int4 *units,
                                 int n_units, bool pairs, int *counter, int C, int n_clusters, int threads,
                                 int ring_pitch, size_t smem_bytes, double *partial, cudaStream_t st,
                                 bool hist)
{
    if (n_units <= 0) return cudaSuccess;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(C * n_clusters, 1, 1);
    cfg.blockDim = dim3(threads, 1, 1);
    cfg.dynamicSmemBytes = smem_bytes;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, resident_fn(R, pairs && !hist, hist), grids_dev, insts, units, n_units, counter,
                              ring_pitch, partial);
}

}  // namespace empso
