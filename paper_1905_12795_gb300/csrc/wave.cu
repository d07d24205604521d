// Acoustic forward modelling of every (model, shot) instance of a generation
// in one persistent launch, with the L2 misfit fused into the time loop
// (section "Testing approach": 2nd order in time, 8th (or 4th) order in space,
// damping layer, Ricker source, receivers along a line, l2 misfit).
//
// Scheme (centred in time, damped, constant density):
//   u^{n+1} = [2 u^n - (1 - t) u^{n-1} + a (lap_h u^n + s^n)] / (1 + t)
// with a = v^2 dt^2, t = (eta_x + eta_z) dt / 2, lap_h the order-2R centred
// Laplacian with zero values outside the padded grid, and s^n the bilinear
// point source r(n dt) b / (hx hz).  Trace sample n is the bilinear sample of
// u^{n+1}; phi = 1/2 sum (d - d_obs)^2.
//
// Work decomposition: a CTA owns one instance at a time, taken from a global
// queue (dynamic, so uneven instance sizes balance); its two wavefield
// buffers live in a private slot of global memory (L2-resident while the
// instance runs).  A thread owns one float4 column group and walks a run of
// rows with the 2R+1 rows of the z-stencil held in registers, so each row
// costs one new centre load plus the left/right float4 neighbours for the
// x-stencil.  u^{n+1} overwrites u^{n-1} in place.  One CTA barrier per step;
// the receivers of u^n are sampled during step n (they only read u^n).
#include "internal.cuh"
#include "stencil.cuh"

namespace empso {

namespace {

struct Corners {
    int k;          // buffer offset of the lower-left corner
    float w[4];     // (i0,j0) (i0+1,j0) (i0,j0+1) (i0+1,j0+1)
};

__device__ __forceinline__ Corners bilinear(float x, float z, const GridDev &g)
{
    float fx = x / g.hx + (float)g.pad;
    float fz = z / g.hz + (float)g.pad;
    int i0 = (int)floorf(fx), j0 = (int)floorf(fz);
    i0 = min(max(i0, 0), g.NX - 2);
    j0 = min(max(j0, 0), g.NZ - 2);
    float ax = fx - (float)i0, az = fz - (float)j0;
    Corners c;
    c.k = (j0 + HALO) * g.pitch + i0 + HALO;
    c.w[0] = (1.f - ax) * (1.f - az);
    c.w[1] = ax * (1.f - az);
    c.w[2] = (1.f - ax) * az;
    c.w[3] = ax * az;
    return c;
}

__device__ __forceinline__ float lane(const float4 &v, int l)
{
    return l == 0 ? v.x : (l == 1 ? v.y : (l == 2 ? v.z : v.w));
}

template <int R, int THREADS>
__device__ void run_instance(const GridDev &g, const Inst &in, float *bufA, float *bufB,
                             double *red, double *partial)
{
    const int tid = threadIdx.x;
    // zero both time levels (interior, halo and alignment columns)
    {
        float4 *z4 = reinterpret_cast<float4 *>(bufA);
        long long n4 = (2 * g.field) / 4;
        for (long long e = tid; e < n4; e += THREADS) z4[e] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    // source corners and per-node weights b / (hx hz)
    const Corners sc = bilinear(in.sx, in.sz, g);
    const int s_j0 = sc.k / g.pitch - HALO, s_i0 = sc.k % g.pitch - HALO;
    const float inv_cell = 1.f / (g.hx * g.hz);

    // thread -> (column group, run of rows)
    const int NQ = g.NQ;
    int nseg = THREADS / NQ;
    if (nseg < 1) nseg = 1;
    if (nseg > g.NZ) nseg = g.NZ;
    const int L = (g.NZ + nseg - 1) / nseg;
    const int items = NQ * nseg;

    float cx[R + 1], cz[R + 1];
#pragma unroll
    for (int m = 0; m <= R; ++m) {
        cx[m] = g.cxm[m];
        cz[m] = g.czm[m];
    }
    const float cres = g.cres;
    double acc = 0.0;
    __syncthreads();

    float *cur = bufA, *prev = bufB;
    for (int n = 0; n <= g.nt; ++n) {
        if (n < g.nt) {
            const float rn = g.wavelet[n] * inv_cell;
            for (int item = tid; item < items; item += THREADS) {
                const int q = item % NQ, seg = item / NQ;
                const int j0 = seg * L;
                const int j1 = min(g.NZ, j0 + L);
                if (j0 >= j1) continue;
                const int col = HALO + 4 * q;
                const float4 exq = *reinterpret_cast<const float4 *>(g.ex + col);
                const bool src_cols = (s_i0 >= 4 * q - 1) && (s_i0 <= 4 * q + 3);
                const bool src_here = src_cols && (s_j0 + 1 >= j0) && (s_j0 < j1);
                float4 w[2 * R + 1];
#pragma unroll
                for (int m = 0; m < 2 * R; ++m)
                    w[m] = *reinterpret_cast<const float4 *>(cur + (size_t)(j0 - R + m + HALO) * g.pitch + col);
                for (int j = j0; j < j1; ++j) {
                    const size_t row = (size_t)(j + HALO) * g.pitch;
                    w[2 * R] = *reinterpret_cast<const float4 *>(cur + row + (size_t)R * g.pitch + col);
                    const float4 lft = *reinterpret_cast<const float4 *>(cur + row + col - 4);
                    const float4 rgt = *reinterpret_cast<const float4 *>(cur + row + col + 4);
                    float4 um = *reinterpret_cast<const float4 *>(prev + row + col);
                    const float4 av = *reinterpret_cast<const float4 *>(in.a + row + col);
                    const float ezj = g.ez[j + HALO];
                    float s[4 * (2 * XGroups<R>::G + 1)];
                    if (XGroups<R>::G == 1) {
                        xline1(lft, w[R], rgt, s);
                    } else {
                        const float4 l2 = *reinterpret_cast<const float4 *>(cur + row + col - 8);
                        const float4 r2 = *reinterpret_cast<const float4 *>(cur + row + col + 8);
                        xline2(l2, lft, w[R], rgt, r2, s);
                    }
                    float2 L01, L23;
                    lap_group<R>(w, s, cx, cz, cres, L01, L23);
                    const float lapv[4] = {L01.x, L01.y, L23.x, L23.y};
                    float outv[4];
#pragma unroll
                    for (int l = 0; l < 4; ++l) {
                        float lap = lapv[l];
                        if (src_here) {
                            const int I = 4 * q + l;
                            float b = 0.f;
                            if (j == s_j0) b += (I == s_i0 ? sc.w[0] : 0.f) + (I == s_i0 + 1 ? sc.w[1] : 0.f);
                            if (j == s_j0 + 1) b += (I == s_i0 ? sc.w[2] : 0.f) + (I == s_i0 + 1 ? sc.w[3] : 0.f);
                            lap = fmaf(b, rn, lap);
                        }
                        const float t = lane(exq, l) + ezj;
                        const float u0 = s[4 * XGroups<R>::G + l];
                        const float num = fmaf(lane(av, l), lap, fmaf(2.f, u0, -(1.f - t) * lane(um, l)));
                        outv[l] = num / (1.f + t);
                    }
                    um = make_float4(outv[0], outv[1], outv[2], outv[3]);
                    *reinterpret_cast<float4 *>(prev + row + col) = um;
#pragma unroll
                    for (int m = 0; m < 2 * R; ++m) w[m] = w[m + 1];
                }
            }
        }
        // receivers sample u^n (record n - 1): `cur` is read-only this step
        if (n >= 1) {
            for (int r = tid; r < in.nrec; r += THREADS) {
                const float2 p = in.rec[r];
                const Corners c = bilinear(p.x, p.y, g);
                const float d = c.w[0] * cur[c.k] + c.w[1] * cur[c.k + 1] +
                                c.w[2] * cur[c.k + g.pitch] + c.w[3] * cur[c.k + g.pitch + 1];
                const size_t o = (size_t)(n - 1) * in.nrec + r;
                if (in.traces) in.traces[o] = d;
                if (in.dobs) {
                    const float e = d - in.dobs[o];
                    acc += (double)e * (double)e;
                }
            }
        }
        __syncthreads();
        float *t = cur;
        cur = prev;
        prev = t;
    }
    // fixed-order block reduction of the residual energy
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((tid & 31) == 0) red[tid >> 5] = acc;
    __syncthreads();
    if (tid < 32) {
        double v = (tid < THREADS / 32) ? red[tid] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (tid == 0) partial[in.out] = 0.5 * v;
    }
    __syncthreads();
}

template <int THREADS>
__global__ void __launch_bounds__(THREADS, 1)
wave_kernel(const GridDev *__restrict__ grids, const Inst *__restrict__ insts, int n_inst,
            int *counter, float *slots, long long slot_floats, double *partial)
{
    __shared__ int s_q;
    __shared__ double red[32];
    __shared__ GridDev sg;
    float *bufA = slots + (size_t)blockIdx.x * slot_floats;
    for (;;) {
        if (threadIdx.x == 0) s_q = atomicAdd(counter, 1);
        __syncthreads();
        const int q = s_q;
        if (q >= n_inst) break;
        const Inst in = insts[q];
        if (threadIdx.x == 0) sg = grids[in.grid];
        __syncthreads();
        const GridDev g = sg;
        float *bufB = bufA + g.field;
        if (g.R == 8) run_instance<8, THREADS>(g, in, bufA, bufB, red, partial);
        else if (g.R == 4) run_instance<4, THREADS>(g, in, bufA, bufB, red, partial);
        else if (g.R == 2) run_instance<2, THREADS>(g, in, bufA, bufB, red, partial);
        else run_instance<1, THREADS>(g, in, bufA, bufB, red, partial);
    }
}

}  // namespace

int wave_max_ctas_per_sm(int threads)
{
    int n = 0;
    if (threads == 512)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, wave_kernel<512>, 512, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, wave_kernel<1024>, 1024, 0);
    return n;
}

cudaError_t launch_wave(const GridDev *grids_dev, const Inst *insts, int n_inst, int *counter,
                        float *slots, long long slot_floats, int n_ctas, int threads,
                        double *partial, cudaStream_t st)
{
    if (n_inst <= 0) return cudaSuccess;
    if (threads == 512)
        wave_kernel<512><<<n_ctas, 512, 0, st>>>(grids_dev, insts, n_inst, counter, slots,
                                                 slot_floats, partial);
    else
        wave_kernel<1024><<<n_ctas, 1024, 0, st>>>(grids_dev, insts, n_inst, counter, slots,
                                                   slot_floats, partial);
    return cudaGetLastError();
}

// misfit[p] = sum_s weight_s partial[p][s] in fixed shot order; non-finite
// sums become +inf and are counted in nf[0] (running) and nf[1] (per call).
__global__ void finalize_kernel(const double *partial, const float *weights, int P, int S,
                                double *misfit, unsigned long long *nf)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    double s = 0.0;
    for (int k = 0; k < S; ++k) s += (double)weights[k] * partial[(size_t)p * S + k];
    if (!isfinite(s)) {
        s = __longlong_as_double(0x7ff0000000000000LL);
        if (nf) {
            atomicAdd(nf, 1ull);
            atomicAdd(nf + 1, 1ull);
        }
    }
    misfit[p] = s;
}

cudaError_t launch_finalize(const double *partial, const float *weights, int P, int S,
                            double *misfit, unsigned long long *nf, cudaStream_t st)
{
    if (P <= 0) return cudaSuccess;
    finalize_kernel<<<(P + 127) / 128, 128, 0, st>>>(partial, weights, P, S, misfit, nf);
    return cudaGetLastError();
}

}  // namespace empso
