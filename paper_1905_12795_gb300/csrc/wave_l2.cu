// L2-resident cluster variant of the persistent modelling launch, for grids
// whose two time levels do not fit the shared memory of a cluster (e.g. the
// 921 x 301 grid at 10 m with a 60-cell damping layer).  Same scheme and
// fused source/receiver/misfit work as the other variants (section "Testing
// approach": 2nd order in time, 4th/8th order in space, damping layer, Ricker
// source, l2 misfit).
//
// A thread-block cluster of C CTAs owns one instance at a time (global
// queue) and splits its rows into C slabs, as the on-chip variant does, but
// both time levels live in a per-cluster buffer in global memory laid out as
// (C rows_c + 2R) rows of NQ + 2 float4 (one zero group each side, R zero rows
// above): a CTA addresses its slab as that buffer plus z0 rows, so the halo
// rows of its neighbours are read in place and nothing is exchanged.  With few
// enough clusters in flight the working set (two levels and the model field,
// ~5 MB per instance of the grid above) stays in the 129 MB L2, so each step
// streams through L2 rather than HBM.  One release/acquire cluster barrier
// per step orders a step's stores before the next step's loads; its acquire
// half also makes the next step's plain (L1-cached) loads see the other SMs'
// stores, so the level being read goes through L1: a float4 that is one
// thread's centre is its neighbours' x-stencil, and the first rows of one run
// of rows are the last rows of the run above, and both come from L1 instead of
// a second L2 read (30.9 -> 21.1 B of L2 traffic per update on the grid
// above).  The level being overwritten is read past L1.  Each thread sweeps
// one run of rows of a float4 column group (plus at most one single row),
// with its z-stencil in a register window and packed FP32x2 arithmetic.
#include <cooperative_groups.h>

#include "internal.cuh"
#include "stencil.cuh"

namespace cg = cooperative_groups;

namespace empso {

namespace {

constexpr int L2_ROWS = 8;
constexpr int L2_NT = 512;
constexpr int L2_CHUNK = 12;  // rows per unrolled chunk of a run (8: 383.2, 12: 389.1 G updates/s on the 921 x 301 grid; 16 spilled)
constexpr int L2_DEPTH = 2;

__device__ __forceinline__ void set_lane(float4 &v, int l, float x)
{
    if (l == 0) v.x = x;
    else if (l == 1) v.y = x;
    else if (l == 2) v.z = x;
    else v.w = x;
}

__device__ __forceinline__ void cp4(void *smem_dst, const void *gsrc)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

__device__ __forceinline__ void bilinear_corner(float x, float z, const GridDev &g, int &i0, int &j0,
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

// with HIST the Laplacian L u^n of every step (without the source term) also
// goes to in.hist (slot n + 1, buffer layout), the history the gradient's
// adjoint pass reads
template <int R, bool HIST>
__device__ void l2_instance(const GridDev &gs, const Inst &in, float4 *U0, float4 *U1, float *wring,
                            float *dring, float4 *rec_w, int *rec_k, int C, int crank,
                            cg::cluster_group &cluster, double *cred, double *wred, double *partial)
{
    const int tid = threadIdx.x, nth = blockDim.x;
    const int NQ = gs.NQ, NZ = gs.NZ, nt = gs.nt, pitch = gs.pitch;
    const float *__restrict__ gex = gs.ex;
    const float *__restrict__ gez = gs.ez;
    const float *__restrict__ gwav = gs.wavelet;
    const int sp4 = NQ + 2;
    const int rows_c = (NZ + C - 1) / C;
    const int z0 = crank * rows_c;
    const int my_rows = max(0, min(NZ, z0 + rows_c) - z0);
    const int brows = C * rows_c + 2 * R;             // rows of each time-level buffer

    // zero this CTA's rows of both levels; rank 0 also the R rows above the
    // grid, the last rank every row below its slab
    {
        const int b0 = crank == 0 ? 0 : R + z0;
        const int b1 = crank == C - 1 ? brows : R + z0 + rows_c;
        const long long n4 = (long long)(b1 - b0) * sp4;
        float4 *p0 = U0 + (long long)b0 * sp4, *p1 = U1 + (long long)b0 * sp4;
        for (long long e = tid; e < n4; e += nth) {
            p0[e] = make_float4(0.f, 0.f, 0.f, 0.f);
            p1[e] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
    float cx[R + 1], cz[R + 1];
#pragma unroll
    for (int m = 0; m <= R; ++m) {
        cx[m] = gs.cxm[m];
        cz[m] = gs.czm[m];
    }
    const float cres = gs.cres;
    int s_i0, s_j0;
    float sw[4];
    bilinear_corner(in.sx, in.sz, gs, s_i0, s_j0, sw);
    const float inv_cell = 1.f / (gs.hx * gs.hz);
    const int nrec = in.nrec;
    const float *__restrict__ dobs = in.dobs;
    // receivers: every CTA samples an equal share [rec_b, rec_e) of them,
    // wherever their rows lie (the time levels are in global memory), so that
    // no CTA holds back the barrier with all of a shot's receivers; rec_k is
    // the corner's float index in a time-level buffer
    const int rec_b = crank * nrec / C, rec_e = (crank + 1) * nrec / C;
    for (int r = rec_b + tid; r < rec_e; r += nth) {
        const float2 pr = in.rec[r];
        int i0, j0;
        float w4[4];
        bilinear_corner(pr.x, pr.y, gs, i0, j0, w4);
        rec_k[r - rec_b] = (j0 + R) * (4 * sp4) + 4 + i0;
        rec_w[r - rec_b] = make_float4(w4[0], w4[1], w4[2], w4[3]);
    }
    if (tid == 0 && nt > 0) cp4(wring, gwav);
    cp_commit();
    cp_wait_all();
    float accf = 0.f;
    double acc = 0.0;
    // Work split: the slab's rows in nseg runs per column group, nseg the
    // smallest count that gives every thread an item, item i = seg NQ + q on
    // thread i (consecutive threads on consecutive groups: coalesced rows).
    // When that makes more items than threads, the last `left` items (the
    // last columns of the last run) are done as single rows, one extra row per
    // thread, so that no thread sweeps more than one run plus one row.  (A
    // loop over 8-row items left a fraction of the threads a whole item more
    // than the rest: 327 G updates/s on the 921 x 301 grid against 375.)
    const int nseg = max(1, min(my_rows, (nth + NQ - 1) / NQ));
    const int items = NQ * nseg, nmain = min(items, nth), left = items - nmain;
    const int r0_last = (nseg - 1) * my_rows / nseg, len_last = my_rows - r0_last;
    const float4 *__restrict__ arow = reinterpret_cast<const float4 *>(in.a + (size_t)HALO * pitch + HALO);
    const int ap4 = pitch / 4;

    cluster.sync();                          // zeroed before any CTA reads a neighbour's rows

    float4 *cur = U0 + (long long)z0 * sp4, *nxt = U1 + (long long)z0 * sp4;
    for (int n = 0; n <= nt; ++n) {
        {
            const int iw = n + 1, ir = n;
            if (tid == 0 && iw < nt) cp4(wring + iw % L2_DEPTH, gwav + iw);
            if (dobs && ir < nt)
                for (int r = rec_b + tid; r < rec_e; r += nth)
                    cp4(dring + (ir % L2_DEPTH) * nrec + r, dobs + (size_t)ir * nrec + r);
            cp_commit();
        }
        // receivers sample u^n (record n - 1) before the sweep, so that their
        // loads overlap the other warps' work instead of delaying the barrier
        if (n >= 1) {
            const float *cf = reinterpret_cast<const float *>(cur - (long long)z0 * sp4);   // the level's buffer
            const int sp = 4 * sp4;
            for (int r = rec_b + tid; r < rec_e; r += nth) {
                const int k0 = rec_k[r - rec_b];
                const float4 w4 = rec_w[r - rec_b];
                const float d = w4.x * __ldcg(cf + k0) + w4.y * __ldcg(cf + k0 + 1) +
                                w4.z * __ldcg(cf + k0 + sp) + w4.w * __ldcg(cf + k0 + sp + 1);
                if (in.traces) in.traces[(size_t)(n - 1) * nrec + r] = d;
                if (dobs) {
                    const float e = d - dring[((n - 1) % L2_DEPTH) * nrec + r];
                    accf = fmaf(e, e, accf);
                }
            }
            if ((n & 31) == 0) {
                acc += (double)accf;
                accf = 0.f;
            }
        }
        if (n < nt) {
            const float rn = wring[n % L2_DEPTH];
            // rows r0 .. r0 + len - 1 of column group q, swept downwards in
            // chunks of L2_CHUNK rows, each with the z-stencil in a register
            // window (its first 2R rows reloaded per chunk, mostly from L1:
            // this thread read them a moment before; carrying the window
            // across chunks made the compiler spill)
            auto sweep = [&](const int q, const int r0, const int len) {
                const float4 ex = __ldg(reinterpret_cast<const float4 *>(gex + HALO) + q);
                const float2 gx01 = make_float2(2.f / (1.f + ex.x), 2.f / (1.f + ex.y));
                const float2 gx23 = make_float2(2.f / (1.f + ex.z), 2.f / (1.f + ex.w));
                const int ks = s_j0 - (z0 + r0);                  // run row of the source's first corner row
                const bool src_here = s_i0 >= 4 * q - 1 && s_i0 <= 4 * q + 3 && ks + 1 >= 0 && ks < len;
                float4 sb0 = make_float4(0.f, 0.f, 0.f, 0.f), sb1 = sb0;
                if (src_here) {
#pragma unroll
                    for (int l = 0; l < 4; ++l) {
                        const int I = 4 * q + l;
                        const float bx0 = (I == s_i0 ? 1.f : 0.f), bx1 = (I == s_i0 + 1 ? 1.f : 0.f);
                        set_lane(sb0, l, (bx0 * sw[0] + bx1 * sw[1]) * inv_cell);
                        set_lane(sb1, l, (bx0 * sw[2] + bx1 * sw[3]) * inv_cell);
                    }
                }
                for (int k0 = 0; k0 < len; k0 += L2_CHUNK) {
                    float4 w[2 * R + 1];
#pragma unroll
                    for (int m = 0; m < 2 * R; ++m) w[m] = *(cur + (r0 + k0 + m) * sp4 + 1 + q);
#pragma unroll
                    for (int j = 0; j < L2_CHUNK; ++j) {
                        const int k = k0 + j;
                        if (k >= len) break;
                        const int lr = R + r0 + k;
                        w[2 * R] = *(cur + (lr + R) * sp4 + 1 + q);
                        const float4 lft = *(cur + lr * sp4 + q);
                        const float4 rgt = *(cur + lr * sp4 + 2 + q);
                        const float4 um = __ldcg(nxt + lr * sp4 + 1 + q);
                        const int zr = z0 + r0 + k;                   // padded row of the output
                        const float4 av = __ldg(arow + (size_t)min(zr, NZ - 1) * ap4 + q);
                        const float2 c01 = lo2(w[R]), c23 = hi2(w[R]);
                        float xs[12];
                        xline1(lft, w[R], rgt, xs);
                        float2 lap01, lap23;
                        lap_group<R>(w, xs, cx, cz, cres, lap01, lap23);
                        const float4 lap_u = make_float4(lap01.x, lap01.y, lap23.x, lap23.y);   // L u^n
                        if (src_here && (k == ks || k == ks + 1)) {
                            const float4 sb = (k == ks) ? sb0 : sb1;
                            lap01 = __ffma2_rn(make_float2(sb.x, sb.y), make_float2(rn, rn), lap01);
                            lap23 = __ffma2_rn(make_float2(sb.z, sb.w), make_float2(rn, rn), lap23);
                        }
                        // u^{n+1} = g (u^n - u^{n-1}) + u^{n-1} + (a f) lap, g = 2 f, f = 1 / (1 + t)
                        const float ezk = zr < NZ ? __ldg(gez + zr + HALO) : 0.f;
                        float2 g01 = gx01, g23 = gx23;
                        if (ezk != 0.f) {
                            g01 = make_float2(__fdividef(2.f, 1.f + (ex.x + ezk)), __fdividef(2.f, 1.f + (ex.y + ezk)));
                            g23 = make_float2(__fdividef(2.f, 1.f + (ex.z + ezk)), __fdividef(2.f, 1.f + (ex.w + ezk)));
                        }
                        const float2 af01 = __fmul2_rn(make_float2(av.x, av.y), __fmul2_rn(g01, make_float2(0.5f, 0.5f)));
                        const float2 af23 = __fmul2_rn(make_float2(av.z, av.w), __fmul2_rn(g23, make_float2(0.5f, 0.5f)));
                        const float2 um01 = make_float2(um.x, um.y), um23 = make_float2(um.z, um.w);
                        const float2 o01 = __ffma2_rn(g01, __fadd2_rn(c01, make_float2(-um.x, -um.y)),
                                                      __ffma2_rn(af01, lap01, um01));
                        const float2 o23 = __ffma2_rn(g23, __fadd2_rn(c23, make_float2(-um.z, -um.w)),
                                                      __ffma2_rn(af23, lap23, um23));
                        nxt[lr * sp4 + 1 + q] = make_float4(o01.x, o01.y, o23.x, o23.y);
                        if (HIST)   // L u^n for the adjoint pass (written once: evict first)
                            __stcs(reinterpret_cast<float4 *>(in.hist + (size_t)(n + 1) * gs.field) +
                                       (size_t)(zr + HALO) * ap4 + HALO4 + q,
                                   lap_u);
#pragma unroll
                        for (int m = 0; m < 2 * R; ++m) w[m] = w[m + 1];
                    }
                }
            };
            if (tid < nmain) {
                const int seg = tid / NQ, r0 = seg * my_rows / nseg;
                sweep(tid % NQ, r0, (seg + 1) * my_rows / nseg - r0);
            }
            for (int e = tid; e < left * len_last; e += nth)
                sweep(NQ - left + e / len_last, r0_last + e % len_last, 1);
        }
        cp_wait_all();
        cluster.sync();
        float4 *t = cur;
        cur = nxt;
        nxt = t;
    }
    if (!dobs) accf = 0.f, acc = 0.0;
    acc += (double)accf;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((tid & 31) == 0) wred[tid >> 5] = acc;
    __syncthreads();
    if (tid < 32) {
        double v = (tid < nth / 32) ? wred[tid] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (tid == 0) *cluster.map_shared_rank(cred + crank, 0) = v;
    }
    cluster.sync();
    if (crank == 0 && tid == 0) {
        double sum = 0.0;
        for (int c = 0; c < C; ++c) sum += cred[c];
        partial[in.out] = 0.5 * sum;
    }
}

template <int R, bool HIST>
__global__ void __launch_bounds__(L2_NT, 1)
wave_l2_kernel(const GridDev *__restrict__ grids, const Inst *__restrict__ insts, int n_inst,
               int *counter, float4 *slots, long long slot_f4, int ring_pitch, double *partial)
{
    extern __shared__ float4 smem4[];
    __shared__ int s_q;
    __shared__ double cred[16];
    __shared__ double wred[L2_NT / 32];
    __shared__ GridDev sg;
    cg::cluster_group cluster = cg::this_cluster();
    const int C = (int)cluster.num_blocks();
    const int crank = (int)cluster.block_rank();
    float4 *U0 = slots + (long long)(blockIdx.x / C) * 2 * slot_f4;
    float4 *U1 = U0 + slot_f4;
    float *wring = reinterpret_cast<float *>(smem4);
    float *dring = wring + 4;
    float4 *rec_w = reinterpret_cast<float4 *>(dring + ((L2_DEPTH * ring_pitch + 3) / 4) * 4);
    int *rec_k = reinterpret_cast<int *>(rec_w + ring_pitch);
    for (;;) {
        if (crank == 0 && threadIdx.x == 0) {
            const int q = atomicAdd(counter, 1);
            for (int c = 0; c < C; ++c) *cluster.map_shared_rank(&s_q, c) = q;
        }
        cluster.sync();
        const int q = s_q;
        if (q >= n_inst) break;
        const Inst in = insts[q];
        if (threadIdx.x == 0) sg = grids[in.grid];
        __syncthreads();
        l2_instance<R, HIST>(sg, in, U0, U1, wring, dring, rec_w, rec_k, C, crank, cluster, cred, wred, partial);
    }
}

using L2Fn = void (*)(const GridDev *, const Inst *, int, int *, float4 *, long long, int, double *);

L2Fn l2_fn(int R, bool hist = false)
{
    if (hist) {
        if (R == 4) return wave_l2_kernel<4, true>;
        if (R == 2) return wave_l2_kernel<2, true>;
        return R == 1 ? wave_l2_kernel<1, true> : nullptr;
    }
    if (R == 4) return wave_l2_kernel<4, false>;
    if (R == 2) return wave_l2_kernel<2, false>;
    return R == 1 ? wave_l2_kernel<1, false> : nullptr;
}

}  // namespace

int l2_max_threads() { return L2_NT; }

size_t l2_smem_bytes(int ring_pitch)
{
    return sizeof(float) * (4 + ((size_t)L2_DEPTH * ring_pitch + 3) / 4 * 4) +
           (sizeof(float4) + sizeof(int)) * (size_t)ring_pitch;
}

// float4 per time-level buffer of grid g on a cluster of C CTAs
long long l2_slot_f4(const GridDev &g, int C)
{
    const int rows_c = (g.NZ + C - 1) / C;
    return (long long)(C * rows_c + 2 * g.R) * (g.NQ + 2);
}

// a cluster of C CTAs runs grid g when no CTA is left without rows and every
// slab holds at least R rows (a slab's window reads stay inside the
// C rows_c + 2R rows of the buffer in any case)
bool l2_fits(const GridDev &g, int C)
{
    const int rows_c = (g.NZ + C - 1) / C;
    return C >= 1 && C <= 16 && rows_c >= L2_ROWS && (C - 1) * rows_c < g.NZ;
}

cudaError_t l2_configure(int R, size_t smem, int C)
{
    cudaError_t e = cudaSuccess;
    for (const bool hist : {false, true}) {
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(l2_fn(R, hist), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess && C > 8)
            e = cudaFuncSetAttribute(l2_fn(R, hist), cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    }
    return e;
}

int l2_max_clusters(int R, int C, int threads, size_t smem, bool hist)
{
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(C * 64, 1, 1);
    cfg.blockDim = dim3(threads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    const cudaError_t e = cudaOccupancyMaxActiveClusters(&n, l2_fn(R, hist), &cfg);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return -(int)e;        // the query's error, negated
    }
    return n;
}

cudaError_t launch_wave_l2(int R, const GridDev *grids_dev, const Inst *insts, int n_inst, int *counter,
                           int C, int n_clusters, int threads, float4 *slots, long long slot_f4,
                           int ring_pitch, size_t smem, double *partial, cudaStream_t st, bool hist)
{
    if (n_inst <= 0) return cudaSuccess;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(C * n_clusters, 1, 1);
    cfg.blockDim = dim3(threads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, l2_fn(R, hist), grids_dev, insts, n_inst, counter, slots, slot_f4,
                              ring_pitch, partial);
}

}  // namespace empso
