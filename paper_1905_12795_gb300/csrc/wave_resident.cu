// On-chip ("resident") variant of the persistent modelling launch: the same
// scheme and fused source/receiver/misfit work as wave.cu (section "Testing
// approach": 2nd order in time, 4th/8th order in space, damping layer, Ricker
// source, l2 misfit), but an instance's two time levels never leave the SMs.
//
// A thread-block cluster of C CTAs owns one instance at a time (taken from a
// global queue by cluster rank 0).  The padded grid is split by rows: CTA c
// holds rows [c*rows_c, (c+1)*rows_c) of u^n and u^{n-1}/u^{n+1} in its shared
// memory with R halo rows above and below, and its slab of the model field
// a = v^2 dt^2 (pre-scaled by the damping).  Every step each thread updates a
// run of at most RW consecutive rows of one float4 column group (z-stencil
// from a register window, x-stencil from the neighbouring float4s in shared
// memory, the next row's inputs read while the current one is computed),
// writes u^{n+1} in place of u^{n-1}, and then copies its slab's first/last R
// rows straight into the halo rows of the neighbouring CTAs (distributed
// shared memory).  One cluster barrier (release/acquire) per step orders it
// all.  Global memory is touched only for the model field (once per
// instance), the observed traces and the output.
//
// Two instantiations of the same code: runs of up to RW = 8 rows per thread
// with up to 512 threads (128 registers), and up to RW = 13 with up to 384
// threads (168 registers); the run length itself (4 .. 13: the number of runs
// a slab is cut into, hence the threads) is a launch parameter, chosen per
// batch by the planner and the autotuner.
#include <cooperative_groups.h>

#include "internal.cuh"
#include "stencil.cuh"

namespace cg = cooperative_groups;

namespace empso {

namespace {

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

// Column groups with a lane in the x-damping layer (columns [0, pad) and
// [NX - pad, NX)): groups [0, qa) and [qb, NQ)
__device__ __forceinline__ void xpad_groups(const GridDev &g, int &qa, int &qb)
{
    qa = min(g.NQ, (g.pad + 3) / 4);
    qb = max(qa, min(g.NQ, (g.NX - g.pad) / 4));
}

// slot of column group q in a row of the damping table: 0 for the groups
// outside the x-damping layer, 1 .. for the others
__device__ __forceinline__ int gslot(int q, int qa, int qb)
{
    return q < qa ? 1 + q : (q >= qb ? 1 + qa + (q - qb) : 0);
}

// Source position of the instance, shared by the CTA: bilinear corner (padded
// indices) and the four weights b / (hx hz)
struct SrcInfo {
    int i0, j0;
    float w[4];
};

// One step of a work item: rows r0 .. r0 + nrows - 1 (nrows <= RW) of column
// group q (cq / nq / mq point at group q of row 0 of u^n, u^{n-1} -> u^{n+1}
// and the pre-scaled model slab).  ZPAD (the same for a whole CTA): some row
// of the slab lies in the z-damping layer, so g comes from the CTA's table
// (gq: the group's column of it, gst float4 per row); otherwise g is the
// per-lane constant gx.  The rows are swept downwards
// (D = 1) or upwards (D = -1, the window mirrored; the stencil is symmetric
// in z), one instruction stream for both.  The first R rows swept are also
// halo rows of a neighbouring CTA when `peer` is set: they go to its buffer
// (shared-row offset peer_off) as soon as they are computed, so the remote
// stores complete under the rest of the sweep.
template <int R, int RW, bool ZPAD, bool HIST>
__device__ __forceinline__ void sweep_item(const float4 *__restrict__ cq, float4 *__restrict__ nq,
                                           const float4 *__restrict__ mq, const float4 *__restrict__ gq,
                                           int gst, int sp4, int NQ, int r0, int nrows, int D, const float *cx,
                                           const float *cz, float cres, float2 gx01, float2 gx23,
                                           float4 *__restrict__ hrow, int hp4, float4 *__restrict__ peer,
                                           int peer_off)
{
    const float2 m1 = splat2(-1.f);
    const int rs = D > 0 ? r0 : r0 + nrows - 1; // first slab row swept
    const int ds = D * sp4, dm = D * NQ, dh = D * hp4;
    const float4 *cp = cq + (R + rs) * sp4;      // u^n group of the current row
    float4 *np = nq + (R + rs) * sp4;            // its u^{n-1} -> u^{n+1}
    const float4 *ap = mq + rs * NQ;             // its model value
    float4 *hp = HIST ? hrow + (rs - r0) * hp4 : nullptr;
    float4 *pp = peer ? peer + (R + rs + peer_off) * sp4 : nullptr;
    float4 w[2 * R + 1];
#pragma unroll
    for (int m = 0; m < 2 * R; ++m) w[m] = cp[(m - R) * ds];
    // the inputs of the next row are read before this row is stored
    // (software pipelined: the loads need not wait behind the store)
    const int dg = D * gst;
    const float4 *gp = ZPAD ? gq + rs * gst : nullptr;   // the row's update weights
    float4 p_w = cp[R * ds], p_l = cp[-1], p_r = cp[1], p_um = *np, p_av = *ap;
    float4 p_g = ZPAD ? *gp : make_float4(0.f, 0.f, 0.f, 0.f);
    // the run's carried z-differences (lap_group_run, in the 13-row shape,
    // whose registers hold them; bit for bit the same Laplacian as
    // lap_group): d_{k-1} = u_k - u_{k-1}, e_{k-1} = u_{k+1} - u_{k-1},
    // e_{k-2} = u_k - u_{k-2} at the first row
    constexpr bool CARRY = RW > 8;
    float2 dm01 = splat2(0.f), dm23 = dm01, e101 = dm01, e123 = dm01, e201 = dm01, e223 = dm01;
    if (CARRY) {
        dm01 = __ffma2_rn(lo2(w[R - 1]), m1, lo2(w[R]));
        dm23 = __ffma2_rn(hi2(w[R - 1]), m1, hi2(w[R]));
    }
    if (CARRY && R >= 2) {
        e101 = __ffma2_rn(lo2(w[R - 1]), m1, lo2(w[R + 1]));
        e123 = __ffma2_rn(hi2(w[R - 1]), m1, hi2(w[R + 1]));
        e201 = __ffma2_rn(lo2(w[R - 2]), m1, lo2(w[R]));
        e223 = __ffma2_rn(hi2(w[R - 2]), m1, hi2(w[R]));
    }
#pragma unroll
    for (int k = 0; k < RW; ++k) {
        if (k >= nrows) break;
        w[2 * R] = p_w;
        const float4 lft = p_l, rgt = p_r, um = p_um, av = p_av;
        const float4 gv = p_g;
        if (k + 1 < RW) {
            p_w = cp[(R + 1) * ds];
            p_l = cp[ds - 1];
            p_r = cp[ds + 1];
            p_um = np[ds];
            p_av = ap[dm];
            if (ZPAD) p_g = gp[(k + 1) * dg];
        }
        const float2 c01 = lo2(w[R]), c23 = hi2(w[R]);
        float xs[12];
        xline1(lft, w[R], rgt, xs);
        float2 lap01, lap23;
        if (CARRY) {
            float2 dk01, dk23, ek01, ek23;
            lap_group_run<R>(w, xs, cx, cz, cres, dm01, dm23, e201, e223, dk01, dk23, ek01, ek23, lap01, lap23);
            dm01 = dk01;
            dm23 = dk23;
            if (R >= 2) {
                e201 = e101;
                e223 = e123;
                e101 = ek01;
                e123 = ek23;
            }
        } else {
            lap_group<R>(w, xs, cx, cz, cres, lap01, lap23);
        }
        // u^{n+1} = [2 u^n - (1 - t) u^{n-1} + a lap] / (1 + t)
        //         = g (u^n - u^{n-1}) + u^{n-1} + (a f) lap,  g = 2 f, f = 1 / (1 + t)
        // (a f is the pre-scaled model slab)
        float2 g01 = gx01, g23 = gx23;
        if (ZPAD) {
            g01 = lo2(gv);
            g23 = hi2(gv);
        }
        const float2 um01 = lo2(um), um23 = hi2(um);
        const float2 o01 = __ffma2_rn(g01, __ffma2_rn(um01, m1, c01), __ffma2_rn(lo2(av), lap01, um01));
        const float2 o23 = __ffma2_rn(g23, __ffma2_rn(um23, m1, c23), __ffma2_rn(hi2(av), lap23, um23));
        const float4 out = make_float4(o01.x, o01.y, o23.x, o23.y);
        *np = out;
        if (k < R && pp) {
            *pp = out;
            pp += ds;
        }
        if (HIST) {   // the gradient's history: L u^n (written once: evict first)
            __stcs(hp, make_float4(lap01.x, lap01.y, lap23.x, lap23.y));
            hp += dh;
        }
        cp += ds;
        np += ds;
        ap += dm;
#pragma unroll
        for (int m = 0; m < 2 * R; ++m) w[m] = w[m + 1];
    }
}

// C CTAs (ranks base .. base + C - 1 of the cluster; crank is the rank among
// them) run instance `in`; with HIST the Laplacian L u^n of every step (the
// source term excluded) also goes to in.hist, slot n + 1
template <int R, int RW, bool HIST>
__device__ void resident_instance(const GridDev &gs, const Inst &in, float4 *A4, float4 *B4,
                                  float4 *M4, float4 *G4, float *wring, float *dring, float4 *rec_w,
                                  int *rec_k, SrcInfo &src, int C, int crank, int base,
                                  cg::cluster_group &cluster, double *cred, double *wred, double *partial,
                                  int run)
{
    const int tid = threadIdx.x;
    const int nth = blockDim.x;
    // scalars of the grid in registers (the descriptor lives in shared memory)
    const int NQ = gs.NQ, NZ = gs.NZ, nt = gs.nt, pitch = gs.pitch;
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
    // some row of the slab in the z-damping layer (rows of the layer are the
    // first and last of the grid, so the slab's end rows tell); the same path
    // for every thread of the CTA
    const bool zpad =
        my_rows > 0 && (__ldg(gez + z0 + HALO) != 0.f || __ldg(gez + z0 + my_rows - 1 + HALO) != 0.f);
    // Such a CTA tabulates g = 2 / (1 + t) of its rows once per instance: per
    // row one value for the column groups outside the x-damping layer (t = t_z
    // there) in slot 0, and one per lane for each group with a lane in it
    // (slots 1 ..), so that its sweep reads g instead of dividing per point.
    int qa, qb;
    xpad_groups(gs, qa, qb);
    const int gst = 1 + qa + (NQ - qb);
    if (zpad)
        for (int e = tid; e < my_rows * gst; e += nth) {
            const int r = e / gst, sl = e % gst;
            const float tz = __ldg(gez + z0 + r + HALO);
            float4 exq = make_float4(0.f, 0.f, 0.f, 0.f);
            if (sl > 0) {
                const int qq = sl - 1 < qa ? sl - 1 : qb + (sl - 1 - qa);
                exq = __ldg(reinterpret_cast<const float4 *>(gex + HALO) + qq);
            }
            G4[e] = make_float4(2.f / (1.f + (exq.x + tz)), 2.f / (1.f + (exq.y + tz)),
                                2.f / (1.f + (exq.z + tz)), 2.f / (1.f + (exq.w + tz)));
        }
    if (tid == 0) {
        int i0, j0;
        float sw[4];
        corners(in.sx, in.sz, gs, i0, j0, sw);
        const float inv_cell = 1.f / (gs.hx * gs.hz);
        src.i0 = i0;
        src.j0 = j0;
#pragma unroll
        for (int c = 0; c < 4; ++c) src.w[c] = sw[c] * inv_cell;
    }

    // work item: column group q and rows [r0, r1) of the slab, the slab's rows
    // split into nseg runs of at most `run` (<= RW) rows each (lengths differ
    // by one at most), item i = seg NQ + q on thread i.  When the launch has fewer
    // threads than items (a multiple of four warps, so that the SM's four
    // schedulers carry equal work), the last `left` items (the last columns
    // of the last run) are split into single rows instead, one extra row on
    // each of the first left * len_last threads.
    const int nseg = (my_rows + run - 1) / run;
    const int items = NQ * nseg;
    const int nmain = min(items, nth);
    const int left = items - nmain;
    const int r0_last = (nseg - 1) * my_rows / nseg, len_last = my_rows - r0_last;
    const bool active = tid < nmain;
    const int q = active ? tid % NQ : 0;
    const int seg = active ? tid / NQ : 0;
    const int r0 = active ? seg * my_rows / nseg : 0;
    const int r1 = active ? (seg + 1) * my_rows / nseg : 0;
    const bool extra = tid < left * len_last;
    const int qe = extra ? NQ - left + tid / len_last : 0;
    const int re = extra ? r0_last + tid % len_last : 0;
    // a launch shape the planner did not mean (leftover items outside the last
    // run, more extra rows than threads, or runs shorter than the R halo rows
    // they hand to a neighbour) would leave rows uncomputed or halos stale:
    // the instance then reports a NaN misfit (the work and barriers run as
    // usual)
    const bool bad_shape = left > NQ || left * len_last > nth || (nseg > 1 && my_rows / nseg < R);

    float4 ex = make_float4(0.f, 0.f, 0.f, 0.f), exe = ex;
    if (active) ex = __ldg(reinterpret_cast<const float4 *>(gex + HALO) + q);
    if (extra) exe = __ldg(reinterpret_cast<const float4 *>(gex + HALO) + qe);
    // update weight g = 2 / (1 + t) of rows without z-damping: per lane,
    // constant over the instance (g = 2 in the interior); hx for the others
    const float2 gx01 = make_float2(2.f / (1.f + ex.x), 2.f / (1.f + ex.y));
    const float2 gx23 = make_float2(2.f / (1.f + ex.z), 2.f / (1.f + ex.w));
    const float2 gxe01 = make_float2(2.f / (1.f + exe.x), 2.f / (1.f + exe.y));
    const float2 gxe23 = make_float2(2.f / (1.f + exe.z), 2.f / (1.f + exe.w));
    // the damping-table columns of the thread's groups
    const float4 *gq = G4 + gslot(q, qa, qb), *gq_e = G4 + gslot(qe, qa, qb);
    float cx[R + 1], cz[R + 1];
#pragma unroll
    for (int m = 0; m <= R; ++m) {
        cx[m] = gs.cxm[m];
        cz[m] = gs.czm[m];
    }
    const float cres = gs.cres;

    // receivers: every CTA samples an equal share of them, receivers
    // [rec_b, rec_e), whichever CTA holds their rows (reading that CTA's u^n through
    // distributed shared memory): one CTA holding all of a shot's receivers
    // would hold back every barrier (461 receivers in one CTA cost 7-10 % of
    // the step).  Per receiver of the share, computed once per instance: the
    // bilinear weights, and the corner's float index in its holder's slab
    // with the holder's rank in the top 8 bits.
    const int nrec = in.nrec;
    const float *__restrict__ dobs = in.dobs;
    const int rec_b = crank * nrec / C, rec_e = (crank + 1) * nrec / C;
    for (int r = rec_b + tid; r < rec_e; r += nth) {
        const float2 pr = in.rec[r];
        int i0, j0;
        float w4[4];
        corners(pr.x, pr.y, gs, i0, j0, w4);
        const int holder = min(j0 / rows_c, C - 1);
        rec_k[r - rec_b] = (holder << 24) | ((j0 - holder * rows_c + R) * (4 * sp4) + 4 + i0);
        rec_w[r - rec_b] = make_float4(w4[0], w4[1], w4[2], w4[3]);
    }
    const bool has_rec = rec_e > rec_b;
    // staging prologue: the wavelet sample of step 0
    if (tid == 0 && nt > 0) cp_async4(wring, gwav);
    cp_async_commit();
    cp_async_wait<0>();
    float accf = 0.f;
    double acc = 0.0;

    cluster.sync();                                      // zeroed everywhere before halo stores

    // The source: the items holding a row of its corners add (a f) b r(t_n) to
    // those points after their rows (u^{n+1} is linear in the source term).
    // sbit: bit c = 1 when corner row s_j0 + c is one of this item's rows and
    // one of the corner columns lies in group q.
    const int s_i0 = src.i0, s_j0 = src.j0;
    unsigned sbit = 0, sbit_e = 0;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        const int rr = s_j0 + c - z0;
        if (active && s_i0 >= 4 * q - 1 && s_i0 <= 4 * q + 3 && rr >= r0 && rr < r1) sbit |= 1u << c;
        if (extra && s_i0 >= 4 * qe - 1 && s_i0 <= 4 * qe + 3 && rr == re) sbit_e |= 1u << c;
    }
    // the item's role: 1 the first run of a CTA with a CTA above (sweeps down,
    // hands its top rows up first), 2 the last of two or more runs of a CTA
    // with a CTA below (sweeps up, hands its bottom rows down first), 0 any
    // other run (sweeps down); tail: the only run of a CTA with a CTA below
    // copies its bottom rows down after the sweep
    const bool has_prev = crank > 0, has_next = crank < C - 1;
    int role = 0;
    bool tail = false;
    if (active) {
        if (nseg > 1 && seg == nseg - 1) role = has_next ? 2 : 0;
        else if (seg == 0) role = has_prev ? 1 : 0;
        tail = nseg == 1 && has_next;
    }

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

    // history: this item's first row in slot n + 1 (advanced one field per step)
    float4 *hrow = nullptr, *hrow_e = nullptr;
    const int hp4 = pitch / 4;
    if (HIST && active)
        hrow = reinterpret_cast<float4 *>(in.hist) + (size_t)(z0 + r0 + HALO) * hp4 + HALO4 + q;
    if (HIST && extra)
        hrow_e = reinterpret_cast<float4 *>(in.hist) + (size_t)(z0 + re + HALO) * hp4 + HALO4 + qe;
    float4 *cur = A4, *nxt = B4;
    int step = 0;
    // The source term of a piece's corner rows (column group qq, corner-row
    // bits sb), added after its sweep; also to a neighbour's halo copy of the
    // row (the history holds L u^n without it)
    auto add_source = [&](int qq, unsigned sb, float4 *nq, const float4 *mq, float4 *pq, float4 *xq) {
        const float rn = wring[step % DEPTH];
        for (int c = 0; c < 2; ++c) {
            if (!((sb >> c) & 1u)) continue;
            const int rr = s_j0 + c - z0, lr = R + rr;
            float4 v = nq[lr * sp4];
            const float4 av = mq[rr * NQ];
            float4 b = make_float4(0.f, 0.f, 0.f, 0.f);
            const float b0 = src.w[2 * c] * rn, b1 = src.w[2 * c + 1] * rn;
#pragma unroll
            for (int l = 0; l < 4; ++l) {
                const int I = 4 * qq + l;
                set_comp(b, l, (I == s_i0 ? b0 : 0.f) + (I == s_i0 + 1 ? b1 : 0.f));
            }
            v = make_float4(fmaf(av.x, b.x, v.x), fmaf(av.y, b.y, v.y), fmaf(av.z, b.z, v.z),
                            fmaf(av.w, b.w, v.w));
            nq[lr * sp4] = v;
            if (pq && rr < R) pq[(lr + rows_c) * sp4] = v;
            if (xq && rr >= rows_c - R) xq[(lr - rows_c) * sp4] = v;
        }
    };
    for (int n = 0; n <= nt; ++n) {
        step = n;
        if (HIST) {
            hrow += gs.field / 4;
            hrow_e += gs.field / 4;
        }
        // stage wavelet sample n + 1 and record n (sampled in step n + 1); their
        // slots were last read in step n - 1, which the previous barrier closed
        {
            const int iw = n + 1, ir = n;
            if (tid == 0 && iw < nt) cp_async4(wring + iw % DEPTH, gwav + iw);
            if (has_rec && dobs && ir < nt)
                for (int r = rec_b + tid; r < rec_e; r += nth)
                    cp_async4(dring + (ir % DEPTH) * nrec + r, dobs + (size_t)ir * nrec + r);
            cp_async_commit();
        }
        // receivers sample u^n (record n - 1) first: u^n is complete since the
        // last barrier and read-only in this step, and the sampling's chain of
        // dependent shared-memory loads then overlaps the other warps' sweeps
        // (at the end of the step it held back the barrier: 461 receivers in
        // one CTA cost 10 % of the step)
        if (has_rec && n >= 1) {
            const float *cf = reinterpret_cast<const float *>(cur);
            const int sp = 4 * sp4;
            for (int r = rec_b + tid; r < rec_e; r += nth) {
                const int kk = rec_k[r - rec_b], holder = kk >> 24, k0 = kk & 0xffffff;
                const float *hf = holder == crank ? cf : cluster.map_shared_rank(cf, base + holder);
                const float4 w4 = rec_w[r - rec_b];
                const float d = w4.x * hf[k0] + w4.y * hf[k0 + 1] + w4.z * hf[k0 + sp] + w4.w * hf[k0 + sp + 1];
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

        if (n < nt && active) {
            const float4 *cq = cur + 1 + q;           // group q of shared row 0
            float4 *nq = nxt + 1 + q;
            const float4 *mq = M4 + q;
            const bool even = (n & 1) == 0;           // nxt is B4 on even steps, A4 on odd
            float4 *pq = has_prev ? (even ? prev_B : prev_A) + 1 + q : nullptr;
            float4 *xq = has_next ? (even ? next_B : next_A) + 1 + q : nullptr;
            // the first run sweeps down and hands its top rows to the CTA above
            // first; the last run sweeps up and hands its bottom rows to the
            // CTA below first; a middle run has no halo rows
            float4 *peer = role == 1 ? pq : (role == 2 ? xq : nullptr);
            const int D = role == 2 ? -1 : 1;
            const int poff = role == 2 ? -rows_c : rows_c;
            if (zpad)
                sweep_item<R, RW, true, HIST>(cq, nq, mq, gq, gst, sp4, NQ, r0, r1 - r0, D, cx, cz, cres, gx01,
                                              gx23, hrow, hp4, peer, poff);
            else
                sweep_item<R, RW, false, HIST>(cq, nq, mq, gq, gst, sp4, NQ, r0, r1 - r0, D, cx, cz, cres, gx01,
                                               gx23, hrow, hp4, peer, poff);
            if (tail)
                for (int rr = max(r0, rows_c - R); rr < r1; ++rr) xq[(R + rr - rows_c) * sp4] = nq[(R + rr) * sp4];
            if (sbit) add_source(q, sbit, nq, mq, pq, xq);
        }
        if (n < nt && extra) {   // the thread's single extra row
            const float4 *cq = cur + 1 + qe;
            float4 *nq = nxt + 1 + qe;
            const float4 *mq = M4 + qe;
            const bool even = (n & 1) == 0;
            float4 *pq = has_prev ? (even ? prev_B : prev_A) + 1 + qe : nullptr;
            float4 *xq = has_next ? (even ? next_B : next_A) + 1 + qe : nullptr;
            float4 *peer = re < R ? pq : (re >= rows_c - R ? xq : nullptr);
            const int poff = re < R ? rows_c : -rows_c;
            if (zpad)
                sweep_item<R, 1, true, HIST>(cq, nq, mq, gq_e, gst, sp4, NQ, re, 1, 1, cx, cz, cres, gxe01,
                                             gxe23, hrow_e, hp4, peer, poff);
            else
                sweep_item<R, 1, false, HIST>(cq, nq, mq, gq_e, gst, sp4, NQ, re, 1, 1, cx, cz, cres, gxe01,
                                              gxe23, hrow_e, hp4, peer, poff);
            if (sbit_e) add_source(qe, sbit_e, nq, mq, pq, xq);
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
    if (bad_shape) acc = __longlong_as_double(0x7ff8000000000000LL);
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
// HIST (never with PAIRS) also writes the history the gradient's adjoint pass
// reads: L u^n of every step n into slot n + 1.  NT threads at
// most: registers per thread are capped so that NT / 128 warps per scheduler
// fit its quarter of the register file.
template <int NT> struct RegCap {
    static constexpr int v = (16384 / (((NT / 32) + 3) / 4 * 32)) / 8 * 8;
};

template <int R, int NT, int RW, bool PAIRS, bool HIST>
__global__ void __launch_bounds__(NT) __maxnreg__(RegCap<NT>::v)
wave_resident_kernel(const GridDev *__restrict__ grids, const Inst *__restrict__ insts,
                     const int4 *__restrict__ units, int n_units, int *counter, int ring_pitch,
                     double *partial, int run)
{
    extern __shared__ float4 smem4[];
    __shared__ int s_q;
    __shared__ double cred[16];
    __shared__ double wred[NT / 32];
    __shared__ GridDev sg;
    __shared__ SrcInfo src;
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
        float4 *G4 = M4 + (size_t)rows_c * sg.NQ;
        float *wring = reinterpret_cast<float *>(G4 + (size_t)rows_c * resident_gtab_width(sg));
        float *dring = wring + 4 * ((DEPTH + 3) / 4);
        float4 *rec_w = reinterpret_cast<float4 *>(dring + (DEPTH * ring_pitch + 3) / 4 * 4);
        int *rec_k = reinterpret_cast<int *>(rec_w + ring_pitch);
        // rows per run: in a launch over several grids (the PAIRS variant),
        // the instance's own when the planner set one (shorter runs that keep
        // more of the launch's threads busy), else the launch's.  A single-grid
        // launch keeps the launch-wide value (reading it per instance cost
        // that launch 0.75 %)
        const int irun = PAIRS && in.run > 0 ? in.run : run;
        resident_instance<R, RW, HIST>(sg, in, A4, B4, M4, G4, wring, dring, rec_w, rec_k, src, Ce, ce,
                                       sub * Ce, cluster, cred, wred, partial, irun);
    }
}

// The two shapes: rows per thread and thread bound
constexpr int RW_A = 8, NT_A = 512;
constexpr int RW_B = 13, NT_B = 384;

// the shape that runs runs of `rows` rows: up to RW_A rows on the 512-thread
// instantiation, more on the 384-thread one
int shape_threads(int rows) { return rows > RW_A ? NT_B : NT_A; }

}  // namespace

int resident_max_threads(int rows) { return shape_threads(rows); }
int resident_default_rows() { return RW_A; }
bool resident_rows_supported(int rows) { return rows >= 4 && rows <= RW_B; }

// Threads of the work items of grid g on C CTAs with runs of at most `rows`
// rows: one per item, or, when that is not a multiple of four warps, the
// multiple of four warps below it with the leftover items (the last columns
// of the last run) done as single extra rows -- so that the SM's four
// schedulers get the same number of warps -- when they fit (at most NQ
// leftover items, at most one extra row per thread).
int resident_threads(const GridDev &g, int C, int rows)
{
    const int rows_c = (g.NZ + C - 1) / C;
    const int nseg = (rows_c + rows - 1) / rows;
    const int items = g.NQ * nseg;
    const int lo = items / 128 * 128;
    const int left = items - lo;
    if (lo > 0 && left > 0 && left <= g.NQ && left * rows <= lo) return lo;
    return (items + 31) / 32 * 32;
}

// two time levels with halo rows, the slab of the model field, its damping
// table, the staging buffers (wavelet samples, observed records) and the
// receiver tables, for shots of up to ring_pitch receivers
size_t resident_smem_bytes(const GridDev &g, int C, int ring_pitch)
{
    const int rows_c = (g.NZ + C - 1) / C;
    return sizeof(float4) * (2 * (size_t)(rows_c + 2 * g.R) * (g.NQ + 2) + (size_t)rows_c * g.NQ +
                             (size_t)rows_c * resident_gtab_width(g)) +
           sizeof(float) * (4 * ((DEPTH + 3) / 4) + ((size_t)DEPTH * ring_pitch + 3) / 4 * 4) +
           (sizeof(float4) + sizeof(int)) * (size_t)ring_pitch;
}

// Does grid g run on a cluster of C CTAs with runs of at most `rows` rows?
// Each CTA needs at least R rows (so halos come from the nearest neighbour
// only), no CTA may be empty, the work items must fit one thread each, and
// the two time levels plus the model slab the shared memory.
bool resident_fits(const GridDev &g, int C, int ring_pitch, size_t smem_limit, int rows)
{
    const int rows_c = (g.NZ + C - 1) / C;
    if (rows_c < g.R || !resident_rows_supported(rows)) return false;
    if ((C - 1) * rows_c >= g.NZ) return false;
    // a slab cut into several runs hands its first R rows up from its first
    // run and its last R rows down from its last run, so every run must hold
    // R rows (in the full slabs and in the last, shorter one)
    for (const int my : {rows_c, g.NZ - (C - 1) * rows_c}) {
        const int nseg = (my + rows - 1) / rows;
        if (nseg > 1 && my / nseg < g.R) return false;
    }
    if (resident_threads(g, C, rows) > shape_threads(rows)) return false;
    return resident_smem_bytes(g, C, ring_pitch) <= smem_limit;
}

// Rows per run for grid g in a launch of `threads` threads with runs of at
// most `rows` rows, on Ce CTAs per instance: the shortest run (most runs per
// column, so the most threads) whose runs all hold R rows in the full and in
// the last slab and whose work items need no more than the launch's threads,
// when that gives more runs than `rows` does; else 0 (the launch's `rows`).
// A small grid in a launch sized for a larger one (uneven batches) then uses
// the threads the larger grid needs instead of leaving most of them idle.
int resident_grid_run(const GridDev &g, int Ce, int threads, int rows)
{
    const int rows_c = (g.NZ + Ce - 1) / Ce;
    const int last = g.NZ - (Ce - 1) * rows_c;
    if (rows_c < 1 || last < 1) return 0;
    const int nseg0 = (rows_c + rows - 1) / rows;
    int best = 0;
    for (int run = rows - 1; run >= g.R; --run) {
        const int nseg = (rows_c + run - 1) / run;
        if (nseg <= nseg0 || (long long)g.NQ * nseg > threads) continue;
        if (nseg > 1 && rows_c / nseg < g.R) continue;
        const int nl = (last + run - 1) / run;
        if (nl > 1 && last / nl < g.R) continue;
        best = run;
    }
    return best;
}

namespace {

using ResidentFn = void (*)(const GridDev *, const Inst *, const int4 *, int, int *, int, double *, int);

template <int NT, int RW>
ResidentFn resident_fn_shape(int R, bool pairs, bool hist)
{
    if (hist) {
        if (R == 4) return wave_resident_kernel<4, NT, RW, false, true>;
        if (R == 2) return wave_resident_kernel<2, NT, RW, false, true>;
        return R == 1 ? wave_resident_kernel<1, NT, RW, false, true> : nullptr;
    }
    if (pairs) {
        if (R == 4) return wave_resident_kernel<4, NT, RW, true, false>;
        if (R == 2) return wave_resident_kernel<2, NT, RW, true, false>;
        return R == 1 ? wave_resident_kernel<1, NT, RW, true, false> : nullptr;
    }
    if (R == 4) return wave_resident_kernel<4, NT, RW, false, false>;
    if (R == 2) return wave_resident_kernel<2, NT, RW, false, false>;
    if (R == 1) return wave_resident_kernel<1, NT, RW, false, false>;
    return nullptr;
}

ResidentFn resident_fn(int R, bool pairs, bool hist, int rows)
{
    return rows > RW_A ? resident_fn_shape<NT_B, RW_B>(R, pairs, hist)
                       : resident_fn_shape<NT_A, RW_A>(R, pairs, hist);
}
}  // namespace

cudaError_t resident_configure(int R, size_t smem_bytes, int C)
{
    for (const int rows : {RW_A, RW_B})
        for (const bool pairs : {false, true})
            for (const bool hist : {false, true}) {
                if (pairs && hist) continue;
                const ResidentFn f = resident_fn(R, pairs, hist, rows);
                cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                     (int)smem_bytes);
                if (e == cudaSuccess && C > 8)
                    e = cudaFuncSetAttribute(f, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
                if (e != cudaSuccess) return e;
            }
    return cudaSuccess;
}

int resident_max_clusters(int R, int C, int threads, size_t smem_bytes, int rows, bool hist)
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
    if (cudaOccupancyMaxActiveClusters(&n, resident_fn(R, false, hist, rows), &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

cudaError_t launch_wave_resident(int R, const GridDev *grids_dev, const Inst *insts, const int4 *units,
                                 int n_units, bool pairs, int *counter, int C, int n_clusters, int threads,
                                 int rows, int ring_pitch, size_t smem_bytes, double *partial,
                                 cudaStream_t st, bool hist)
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
    return cudaLaunchKernelEx(&cfg, resident_fn(R, pairs && !hist, hist, rows), grids_dev, insts, units,
                              n_units, counter, ring_pitch, partial, rows);
}

}  // namespace empso
