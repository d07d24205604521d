// Elitist-mutated PSO on the device (section "Theory": Eq. 1-3 and the
// elitist-mutation figure; "Testing approach": box constraint, NM, p_em).
//
// This translation unit is compiled with -fmad=false: every FP64 operation is
// a single IEEE-rounded operation in source order, and the transcendental
// functions the method needs (log and cos for Box-Muller normals) are written
// here from their series, so the same inputs give the same bits on any IEEE
// machine that evaluates the same sequence.
#include <algorithm>

#include "internal.cuh"

namespace empso {

namespace {

enum { INIT_X = 0, INIT_V = 1, RU1 = 2, RU2 = 3, EM_U = 4, EM_N = 5 };

// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): ten rounds of two
// 32x32->64 multiplications with the key advanced by the Weyl increments
// 0x9E3779B9 / 0xBB67AE85 between rounds.
__device__ __forceinline__ uint4 philox(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

__device__ __forceinline__ uint4 draw(uint64_t seed, uint32_t k, uint32_t i, uint32_t d,
                                      uint32_t purpose)
{
    return philox(make_uint4(k, i, d, purpose), (uint32_t)seed, (uint32_t)(seed >> 32));
}

// open-interval uniform: w / 2^32 + 1 / 2^33
__device__ __forceinline__ double unit(uint32_t w)
{
    return (double)w * 2.3283064365386962890625e-10 + 1.16415321826934814453125e-10;
}

// ln u = e ln 2 + 2 atanh((m - 1) / (m + 1)), u = m 2^e, m in [sqrt(1/2), sqrt(2));
// atanh by its odd power series through s^23.
__device__ double series_log(double u)
{
    int e;
    double m = frexp(u, &e);
    if (m < 0.70710678118654752440) {
        m = m * 2.0;
        e = e - 1;
    }
    const double s = (m - 1.0) / (m + 1.0);
    const double s2 = s * s;
    double p = 1.0 / 23.0;
    p = p * s2 + 1.0 / 21.0;
    p = p * s2 + 1.0 / 19.0;
    p = p * s2 + 1.0 / 17.0;
    p = p * s2 + 1.0 / 15.0;
    p = p * s2 + 1.0 / 13.0;
    p = p * s2 + 1.0 / 11.0;
    p = p * s2 + 1.0 / 9.0;
    p = p * s2 + 1.0 / 7.0;
    p = p * s2 + 1.0 / 5.0;
    p = p * s2 + 1.0 / 3.0;
    p = p * s2 + 1.0;
    return (double)e * 0.69314718055994530942 + 2.0 * s * p;
}

// Maclaurin series of cos (through x^20) and sin (through x^21), |x| <= pi/4.
__device__ double cos_poly(double x)
{
    const double x2 = x * x;
    double p = 1.0 / 2432902008176640000.0;
    p = -p * x2 + 1.0 / 6402373705728000.0;
    p = -p * x2 + 1.0 / 20922789888000.0;
    p = -p * x2 + 1.0 / 87178291200.0;
    p = -p * x2 + 1.0 / 479001600.0;
    p = -p * x2 + 1.0 / 3628800.0;
    p = -p * x2 + 1.0 / 40320.0;
    p = -p * x2 + 1.0 / 720.0;
    p = -p * x2 + 1.0 / 24.0;
    p = -p * x2 + 1.0 / 2.0;
    p = -p * x2 + 1.0;
    return p;
}

__device__ double sin_poly(double x)
{
    const double x2 = x * x;
    double p = 1.0 / 51090942171709440000.0;
    p = -p * x2 + 1.0 / 121645100408832000.0;
    p = -p * x2 + 1.0 / 355687428096000.0;
    p = -p * x2 + 1.0 / 1307674368000.0;
    p = -p * x2 + 1.0 / 6227020800.0;
    p = -p * x2 + 1.0 / 39916800.0;
    p = -p * x2 + 1.0 / 362880.0;
    p = -p * x2 + 1.0 / 5040.0;
    p = -p * x2 + 1.0 / 120.0;
    p = -p * x2 + 1.0 / 6.0;
    p = -p * x2 + 1.0;
    return x * p;
}

// cos(2 pi t), t in (0, 1): fold to t in [0, 1/4] by the exact maps
// t -> 1 - t and t -> 1/2 - t (sign flip), then cos or the complementary sin.
__device__ double cos_turns(double t)
{
    double sign = 1.0;
    if (t > 0.5) t = 1.0 - t;
    if (t > 0.25) {
        t = 0.5 - t;
        sign = -1.0;
    }
    const double twopi = 6.28318530717958647693;
    const double r = (t > 0.125) ? sin_poly((0.25 - t) * twopi) : cos_poly(t * twopi);
    return sign * r;
}

__device__ __forceinline__ double uniform_at(uint64_t seed, uint32_t k, uint32_t i, uint32_t d,
                                             uint32_t purpose)
{
    return unit(draw(seed, k, i, d, purpose).x);
}

// Box-Muller from words 0 and 1 of one Philox block
__device__ double normal_at(uint64_t seed, uint32_t k, uint32_t i, uint32_t d)
{
    const uint4 w = draw(seed, k, i, d, EM_N);
    const double u1 = unit(w.x), u2 = unit(w.y);
    return sqrt(-2.0 * series_log(u1)) * cos_turns(u2);
}

__device__ __forceinline__ double clampd(double x, double lo, double hi)
{
    return x < lo ? lo : (x > hi ? hi : x);
}

__global__ void pso_init_kernel(PsoDev s, float *particles_out)
{
    const long long n = (long long)s.P * s.D;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e / s.D), d = (int)(e % s.D);
        const double vr = s.xmax[d] - s.xmin[d];
        const double vm = s.lambda * vr;
        const double ux = uniform_at(s.seed, 0, i, d, INIT_X);
        const double uv = uniform_at(s.seed, 0, i, d, INIT_V);
        const double x = s.xmin[d] + ux * vr;
        s.x[e] = x;
        s.v[e] = vm * (2.0 * uv - 1.0);
        s.p[e] = x;
        s.xf[e] = (float)x;
        if (particles_out) particles_out[e] = (float)x;
        if (d == 0) {
            s.pf[i] = __longlong_as_double(0x7ff0000000000000LL);
            s.order[i] = i;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        s.gk[0] = 0;
        s.gk[1] = 0;
    }
}

constexpr int STEP_THREADS = 1024;

// (key, index) lexicographic order: ties go to the lower index, which makes
// the bitonic sort equivalent to a stable sort of the keys.
__device__ __forceinline__ bool before(double fa, int ia, double fb, int ib)
{
    return fa < fb || (fa == fb && ia < ib);
}

// One generation, first part, in one CTA: personal bests, global best and the
// EM sort; the rank of every particle goes to s.rank_of for the second part.
__global__ void __launch_bounds__(STEP_THREADS)
pso_rank_kernel(PsoDev s, const double *misfit, const double *rank)
{
    __shared__ double key[MAX_PSO_P];
    __shared__ int idx[MAX_PSO_P];
    __shared__ double bf[STEP_THREADS / 32];
    __shared__ int bi[STEP_THREADS / 32];
    const int tid = threadIdx.x;
    const int P = s.P, D = s.D;
    const double inf = __longlong_as_double(0x7ff0000000000000LL);
    const int k = s.gk[1] + 1;

    // 1-2. fitness (non-finite -> +inf) and strict personal-best update
    int N = 1;
    while (N < P) N <<= 1;
    for (int i = tid; i < N; i += STEP_THREADS) {
        if (i < P) {
            double f = misfit[i];
            if (!isfinite(f)) f = inf;
            // EM sort key: the fitness, or the given rank key (surrogate pre-screen)
            double r = rank ? rank[i] : misfit[i];
            if (!isfinite(r)) r = inf;
            key[i] = r;
            idx[i] = i;
            if (f < s.pf[i]) {
                s.pf[i] = f;
                for (int d = 0; d < D; ++d) s.p[(size_t)i * D + d] = s.x[(size_t)i * D + d];
            }
        } else {
            key[i] = inf;
            idx[i] = 0x7fffffff;
        }
    }
    __syncthreads();

    // 3. global best: lowest-index argmin of pf
    double bv = inf;
    int bj = 0x7fffffff;
    for (int i = tid; i < P; i += STEP_THREADS) {
        const double v = s.pf[i];
        if (before(v, i, bv, bj)) {
            bv = v;
            bj = i;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_down_sync(0xffffffffu, bv, o);
        const int oj = __shfl_down_sync(0xffffffffu, bj, o);
        if (before(ov, oj, bv, bj)) {
            bv = ov;
            bj = oj;
        }
    }
    if ((tid & 31) == 0) {
        bf[tid >> 5] = bv;
        bi[tid >> 5] = bj;
    }
    __syncthreads();
    if (tid == 0) {
        double v = bf[0];
        int j = bi[0];
        for (int w = 1; w < STEP_THREADS / 32; ++w)
            if (before(bf[w], bi[w], v, j)) {
                v = bf[w];
                j = bi[w];
            }
        // all-infinite pf: every index ties, the lowest one wins (every
        // thread read gk before the barrier above)
        s.gk[0] = (j == 0x7fffffff) ? 0 : j;
        s.gk[1] = k;
    }

    // 4. EM: stable ascending sort of the fitness (bitonic on (f, i) pairs)
    const bool em = s.em_enabled && k >= s.em_start && s.NM > 0;
    if (em) {
        for (int size = 2; size <= N; size <<= 1) {
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                for (int t = tid; t < N / 2; t += STEP_THREADS) {
                    const int lo = 2 * t - (t & (stride - 1));
                    const int hi = lo + stride;
                    const bool up = (lo & size) == 0;
                    const bool swap = up ? before(key[hi], idx[hi], key[lo], idx[lo])
                                         : before(key[lo], idx[lo], key[hi], idx[hi]);
                    if (swap) {
                        const double tk = key[lo];
                        key[lo] = key[hi];
                        key[hi] = tk;
                        const int ti = idx[lo];
                        idx[lo] = idx[hi];
                        idx[hi] = ti;
                    }
                }
                __syncthreads();
            }
        }
        for (int r = tid; r < P; r += STEP_THREADS) {
            s.rank_of[idx[r]] = r;
            s.order[r] = idx[r];
        }
    } else {
        for (int r = tid; r < P; r += STEP_THREADS) {
            s.rank_of[r] = 0;
            s.order[r] = r;
        }
    }
}

// One generation, second part, one thread per (particle, node) over the whole
// GPU: EM on the NM worst, Eq. 1 / Eq. 2 with clamps on the rest.  Every
// element's arithmetic is independent of the others', so spreading them over
// CTAs changes no bit of the result.
__global__ void pso_move_kernel(PsoDev s, float *particles_out)
{
    const int P = s.P, D = s.D;
    const int g = s.gk[0], k = s.gk[1];
    const int NM = s.NM;
    const bool em = s.em_enabled && k >= s.em_start && NM > 0;
    const double phi = s.c1 + s.c2;
    const double chi = 2.0 / fabs(2.0 - phi - sqrt(phi * phi - 4.0 * phi));
    const double *gx = s.p + (size_t)g * D;
    const long long total = (long long)P * D;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e / D), d = (int)(e % D);
        const double lo = s.xmin[d], hi = s.xmax[d];
        const double vr = hi - lo;
        double x;
        if (em && s.rank_of[i] >= P - NM) {
            const double u = uniform_at(s.seed, k, i, d, EM_U);
            double xn;
            if (u < s.p_em) xn = gx[d] + 0.1 * vr * normal_at(s.seed, k, i, d);
            else xn = gx[d];
            x = clampd(xn, lo, hi);
        } else {
            const double vm = s.lambda * vr;
            const double u1 = uniform_at(s.seed, k, i, d, RU1);
            const double u2 = uniform_at(s.seed, k, i, d, RU2);
            const double xi = s.x[e];
            double vn = chi * (s.v[e] + s.c1 * u1 * (s.p[e] - xi) + s.c2 * u2 * (gx[d] - xi));
            vn = clampd(vn, -vm, vm);
            s.v[e] = vn;
            x = clampd(xi + vn, lo, hi);
        }
        s.x[e] = x;
        s.xf[e] = (float)x;
        if (particles_out) particles_out[e] = (float)x;
    }
}

}  // namespace

cudaError_t launch_pso_init(const PsoDev &s, float *particles_out, cudaStream_t st)
{
    long long n = (long long)s.P * s.D;
    int blocks = (int)((n + 255) / 256);
    if (blocks > 1024) blocks = 1024;
    if (blocks < 1) blocks = 1;
    pso_init_kernel<<<blocks, 256, 0, st>>>(s, particles_out);
    return cudaGetLastError();
}

__global__ void xf_from_x_kernel(PsoDev s)
{
    const long long n = (long long)s.P * s.D;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x)
        s.xf[e] = (float)s.x[e];
}

cudaError_t launch_xf_from_x(const PsoDev &s, cudaStream_t st)
{
    long long n = (long long)s.P * s.D;
    int blocks = (int)std::min<long long>((n + 255) / 256, 1024);
    xf_from_x_kernel<<<blocks < 1 ? 1 : blocks, 256, 0, st>>>(s);
    return cudaGetLastError();
}

cudaError_t launch_pso_step(const PsoDev &s, const double *misfit, float *particles_out,
                            cudaStream_t st, const double *rank)
{
    pso_rank_kernel<<<1, STEP_THREADS, 0, st>>>(s, misfit, rank);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // one element per thread, 256 threads a CTA (P D <= 2048 x 1024 elements)
    const long long n = (long long)s.P * s.D;
    const int blocks = (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, 8192));
    pso_move_kernel<<<blocks, 256, 0, st>>>(s, particles_out);
    return cudaGetLastError();
}

}  // namespace empso
