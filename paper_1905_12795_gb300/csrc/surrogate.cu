// Surrogate network that pre-screens EMPSO particles (the paper has none; it
// serves the pre-screening pattern the library adds): a K -> H -> H -> 1
// ReLU perceptron predicting the standardised log-misfit of a particle from
// its control nodes scaled to [-1, 1].  Dense layers run on the tensor cores
// (BF16 operands, FP32 accumulation), master weights and Adam moments are
// FP32, and the training set is a device-side replay buffer filled with the
// (particle, misfit) pairs the fitness evaluation produces.
#include <cuda_bf16.h>

#include "internal.cuh"

namespace empso {

namespace {

// ---------------------------------------------------------------------------
// C[M][N] = sum_k A(m, k) B(k, n) (+ bias[n], ReLU) with BF16 operands and
// FP32 accumulation on mma.sync m16n8k16.  A(m, k) = A[m lda + k] (a_mk) or
// A[k lda + m]; B(k, n) = B[n ldb + k] (b_nk) or B[k ldb + n].  Tiles of
// 64 x 64 per 128-thread block, 32-deep k-steps staged in shared memory
// (zero-filled past M, N, K).  Outputs: FP32 Cf and/or BF16 Cb.
// ---------------------------------------------------------------------------
constexpr int GBM = 64, GBN = 64, GBK = 32, GPAD = 8;

__device__ __forceinline__ void mma_bf16(float c[4], const unsigned a[4], const unsigned b[2])
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, "
        "{%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__global__ void __launch_bounds__(128)
gemm_bf16_kernel(int M, int N, int K, const __nv_bfloat16 *__restrict__ A, int lda, int a_mk,
                 const __nv_bfloat16 *__restrict__ B, int ldb, int b_nk,
                 const float *__restrict__ bias, int relu, float *Cf, int ldc, __nv_bfloat16 *Cb,
                 int ldcb)
{
    __shared__ __align__(16) __nv_bfloat16 As[GBM][GBK + GPAD];   // (m, k)
    __shared__ __align__(16) __nv_bfloat16 Bs[GBN][GBK + GPAD];   // (n, k)
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int g = lane >> 2, t = lane & 3;
    const int m0 = blockIdx.y * GBM, n0 = blockIdx.x * GBN;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.f;
    const __nv_bfloat16 zero = __float2bfloat16(0.f);
    for (int k0 = 0; k0 < K; k0 += GBK) {
        for (int e = tid; e < GBM * GBK; e += 128) {
            int mm, kk;
            if (a_mk) { mm = e / GBK; kk = e % GBK; } else { kk = e / GBM; mm = e % GBM; }
            const int m = m0 + mm, k = k0 + kk;
            __nv_bfloat16 v = zero;
            if (m < M && k < K) v = a_mk ? A[(size_t)m * lda + k] : A[(size_t)k * lda + m];
            As[mm][kk] = v;
        }
        for (int e = tid; e < GBN * GBK; e += 128) {
            int nn, kk;
            if (b_nk) { nn = e / GBK; kk = e % GBK; } else { kk = e / GBN; nn = e % GBN; }
            const int n = n0 + nn, k = k0 + kk;
            __nv_bfloat16 v = zero;
            if (n < N && k < K) v = b_nk ? B[(size_t)n * ldb + k] : B[(size_t)k * ldb + n];
            Bs[nn][kk] = v;
        }
        __syncthreads();
#pragma unroll
        for (int ks = 0; ks < GBK; ks += 16) {
            unsigned af[2][4], bf[4][2];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int r = wm + 16 * i + g;
                af[i][0] = *reinterpret_cast<const unsigned *>(&As[r][ks + 2 * t]);
                af[i][1] = *reinterpret_cast<const unsigned *>(&As[r + 8][ks + 2 * t]);
                af[i][2] = *reinterpret_cast<const unsigned *>(&As[r][ks + 2 * t + 8]);
                af[i][3] = *reinterpret_cast<const unsigned *>(&As[r + 8][ks + 2 * t + 8]);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int c = wn + 8 * j + g;
                bf[j][0] = *reinterpret_cast<const unsigned *>(&Bs[c][ks + 2 * t]);
                bf[j][1] = *reinterpret_cast<const unsigned *>(&Bs[c][ks + 2 * t + 8]);
            }
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], af[i], bf[j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int m = m0 + wm + 16 * i + g + (e >= 2 ? 8 : 0);
                const int n = n0 + wn + 8 * j + 2 * t + (e & 1);
                if (m >= M || n >= N) continue;
                float v = acc[i][j][e];
                if (bias) v += bias[n];
                if (relu) v = fmaxf(v, 0.f);
                if (Cf) Cf[(size_t)m * ldc + n] = v;
                if (Cb) Cb[(size_t)m * ldcb + n] = __float2bfloat16(v);
            }
}

// ---------------------------------------------------------------------------
// The same product on the 5th-generation tensor cores: tcgen05.mma with BF16
// operands from shared memory and the FP32 accumulator in tensor memory.
// One CTA (4 warps) computes a 128 x NT tile (NT = 64, or N rounded up to 16
// when N < 64) over 64-deep k-chunks, double-buffered: while the tensor core
// works on chunk c, the threads stage chunk c + 1 into the other buffer.
// Staging writes the K-major canonical layout without swizzle (8-row x
// 16-byte core matrices; the two 8-element halves of a 16-deep k-slice 128
// bytes apart, successive 8-row groups 256 bytes apart): rows stored k-fastest
// are copied 16 bytes at a time, operands stored m/n-fastest are transposed
// in registers 8 x 8 elements at a time.  One thread issues four
// 128 x NT x 16 MMAs per chunk and commits them to the buffer's mbarrier;
// after the last chunk every warp reads its 32 accumulator rows with
// tcgen05.ld for the epilogue (bias, ReLU, FP32 and/or BF16 stores).
// ---------------------------------------------------------------------------
constexpr int TM = 128, TKC = 64, TNT = 64;
constexpr int TC_SMEM = 2 * (TKC / 16) * (TM + TNT) * 32;   // two k-chunk buffers

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

// no-swizzle K-major descriptor: start >> 4, LBO (k-direction core stride) >> 4,
// SBO (m/n-direction core stride) >> 4, descriptor version 1
__device__ __forceinline__ unsigned long long umma_desc(const void *p, unsigned lbo, unsigned sbo)
{
    unsigned long long d = 0;
    d |= (unsigned long long)((smem_u32(p) >> 4) & 0x3FFF);
    d |= (unsigned long long)((lbo >> 4) & 0x3FFF) << 16;
    d |= (unsigned long long)((sbo >> 4) & 0x3FFF) << 32;
    d |= 1ull << 46;
    return d;
}

// kind::f16 instruction descriptor: D FP32, A and B BF16, both K-major,
// N >> 3 at bit 17, M >> 4 at bit 24
__device__ __forceinline__ unsigned umma_idesc(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(N >> 3) << 17) | ((unsigned)(M >> 4) << 24);
}

// byte offset of element (row r, k) inside a 16-deep k-slice of a K-major tile
__device__ __forceinline__ int canon_off(int r, int k)
{
    return (r >> 3) * 256 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

__device__ __forceinline__ bool mbar_try(unsigned addr, unsigned parity)
{
    unsigned ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                 " selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok)
                 : "r"(addr), "r"(parity)
                 : "memory");
    return ok != 0;
}

// wait (at most WAIT_LIMIT_NS) for the phase of `parity` of an mbarrier
__device__ __forceinline__ bool mbar_wait_tc(unsigned addr, unsigned parity)
{
    if (mbar_try(addr, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (;;) {
        if (mbar_try(addr, parity)) return true;
        if (global_ns() - t0 > WAIT_LIMIT_NS) return false;
    }
}

// Stage rows r0 .. r0 + R - 1 (of M) x k-chunk k0 .. k0 + 63 (of K) of an
// operand into the canonical layout at dst (4 slices of R x 16 elements).
// kmajor: element (r, k) at src[r ld + k]; otherwise at src[k ld + r].
// vec: ld % 8 == 0 and src 16-byte aligned (16-byte accesses allowed).
__device__ __forceinline__ void stage_operand(unsigned char *dst, const __nv_bfloat16 *__restrict__ src,
                                              int ld, int kmajor, bool vec, int r0, int R, int M,
                                              int k0, int K)
{
    const int tid = threadIdx.x;
    const __nv_bfloat16 zero = __float2bfloat16(0.f);
    if (vec && kmajor) {
        // one 16-byte vector = 8 consecutive k of one row
        for (int v = tid; v < R * (TKC / 8); v += blockDim.x) {
            const int r = v / (TKC / 8), kv = (v % (TKC / 8)) * 8;
            const int row = r0 + r, k = k0 + kv;
            uint4 val = make_uint4(0u, 0u, 0u, 0u);
            if (row < M) {
                const __nv_bfloat16 *p = src + (size_t)row * ld + k;
                if (k + 8 <= K) {
                    val = *reinterpret_cast<const uint4 *>(p);
                } else if (k < K) {
                    __nv_bfloat16 t[8];
                    for (int e = 0; e < 8; ++e) t[e] = (k + e < K) ? p[e] : zero;
                    val = *reinterpret_cast<const uint4 *>(t);
                }
            }
            *reinterpret_cast<uint4 *>(dst + (kv >> 4) * (R * 32) + canon_off(r, kv & 15)) = val;
        }
    } else if (vec && (M & 7) == 0) {
        // 8 (rows) x 8 (k) blocks: eight 16-byte loads along the rows, a
        // register transpose, eight 16-byte stores along k
        for (int b = tid; b < (R / 8) * (TKC / 8); b += blockDim.x) {
            const int rb = (b % (R / 8)) * 8, kb = (b / (R / 8)) * 8;
            const int row = r0 + rb;
            uint4 in[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int k = k0 + kb + i;
                in[i] = (row < M && k < K)
                            ? *reinterpret_cast<const uint4 *>(src + (size_t)k * ld + row)
                            : make_uint4(0u, 0u, 0u, 0u);
            }
            // word j of in[i] holds rows (2j, 2j+1) at k = i; word i of out[m]
            // must hold k = (2i, 2i+1) at row m
            unsigned o[8][4];
            const unsigned *w = reinterpret_cast<const unsigned *>(in);
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const unsigned a = w[(2 * i) * 4 + j], c = w[(2 * i + 1) * 4 + j];
                    o[2 * j][i] = __byte_perm(a, c, 0x5410);
                    o[2 * j + 1][i] = __byte_perm(a, c, 0x7632);
                }
#pragma unroll
            for (int m = 0; m < 8; ++m)
                *reinterpret_cast<uint4 *>(dst + (kb >> 4) * (R * 32) + canon_off(rb + m, kb & 15)) =
                    make_uint4(o[m][0], o[m][1], o[m][2], o[m][3]);
        }
    } else {
        for (int e = tid; e < R * TKC; e += blockDim.x) {
            int r, kk;
            if (kmajor) { r = e / TKC; kk = e % TKC; } else { kk = e / R; r = e % R; }
            const int row = r0 + r, k = k0 + kk;
            __nv_bfloat16 v = zero;
            if (row < M && k < K) v = kmajor ? src[(size_t)row * ld + k] : src[(size_t)k * ld + row];
            *reinterpret_cast<__nv_bfloat16 *>(dst + (kk >> 4) * (R * 32) + canon_off(r, kk & 15)) = v;
        }
    }
}

__global__ void __launch_bounds__(128)
gemm_tc_kernel(int M, int N, int K, const __nv_bfloat16 *__restrict__ A, int lda, int a_mk, int a_vec,
               const __nv_bfloat16 *__restrict__ B, int ldb, int b_nk, int b_vec,
               const float *__restrict__ bias, int relu, float *Cf, int ldc, __nv_bfloat16 *Cb,
               int ldcb, int NT, int *err)
{
    extern __shared__ __align__(1024) unsigned char tsm[];
    __shared__ __align__(8) unsigned long long mbar[2];
    __shared__ unsigned tmem_base;
    __shared__ int s_fail;
    const int stage_bytes = (TKC / 16) * (TM + NT) * 32;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int m0 = blockIdx.y * TM, n0 = blockIdx.x * NT;
    const unsigned ncols = NT <= 32 ? 32u : 64u;        // tensor-memory columns (power of 2)
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&mbar[0])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&mbar[1])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        s_fail = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                         smem_u32(&tmem_base)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const unsigned tmem = tmem_base;
    const unsigned idesc = umma_idesc(TM, NT);
    const int nchunks = (K + TKC - 1) / TKC;
    for (int c = 0; c < nchunks; ++c) {
        const int buf = c & 1;
        unsigned char *As = tsm + buf * stage_bytes;
        unsigned char *Bs = As + (TKC / 16) * TM * 32;
        // the MMAs that read this buffer two chunks ago are done before it is restaged
        if (c >= 2 && !mbar_wait_tc(smem_u32(&mbar[buf]), ((c - 2) >> 1) & 1)) s_fail = 1;
        stage_operand(As, A, lda, a_mk, a_vec != 0, m0, TM, M, c * TKC, K);
        stage_operand(Bs, B, ldb, b_nk, b_vec != 0, n0, NT, N, c * TKC, K);
        // thread-written shared memory -> visible to the tensor core (async proxy)
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            for (int s = 0; s < TKC / 16; ++s) {
                const unsigned long long ad = umma_desc(As + s * (TM * 32), 128, 256);
                const unsigned long long bd = umma_desc(Bs + s * (NT * 32), 128, 256);
                const unsigned acc = (c > 0 || s > 0) ? 1u : 0u;
                asm volatile("{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
                             " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                             "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                             : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                             smem_u32(&mbar[buf]))
                         : "memory");
        }
    }
    // the last commit covers every MMA issued before it
    {
        const int c = nchunks - 1;
        if (!mbar_wait_tc(smem_u32(&mbar[c & 1]), (c >> 1) & 1)) s_fail = 1;
    }
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    __syncthreads();
    // epilogue: warp w reads accumulator rows 32 w .. 32 w + 31 (TMEM lanes)
    const int row = m0 + 32 * warp + (tid & 31);
    const bool fail = s_fail != 0;
    for (int c0 = 0; c0 < NT; c0 += 16) {
        unsigned r[16];
        const unsigned taddr = tmem + ((unsigned)(32 * warp) << 16) + (unsigned)c0;
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
                     : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                       "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
                       "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                     : "r"(taddr)
                     : "memory");
        asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
        if (row >= M || fail) continue;
        const int nb = n0 + c0;
        float v[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            float t = __uint_as_float(r[j]);
            if (bias && nb + j < N) t += bias[nb + j];
            if (relu) t = fmaxf(t, 0.f);
            v[j] = t;
        }
        if (nb + 16 <= N && c0 + 16 <= NT) {
            if (Cf) {
                float *o = Cf + (size_t)row * ldc + nb;
                if ((ldc & 3) == 0 && ((size_t)Cf & 15) == 0) {
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        reinterpret_cast<float4 *>(o)[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                } else {
                    for (int j = 0; j < 16; ++j) o[j] = v[j];
                }
            }
            if (Cb) {
                __nv_bfloat16 *o = Cb + (size_t)row * ldcb + nb;
                if ((ldcb & 7) == 0 && ((size_t)Cb & 15) == 0) {
                    __nv_bfloat162 h[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) h[q] = __floats2bfloat162_rn(v[2 * q], v[2 * q + 1]);
                    reinterpret_cast<uint4 *>(o)[0] = *reinterpret_cast<uint4 *>(&h[0]);
                    reinterpret_cast<uint4 *>(o)[1] = *reinterpret_cast<uint4 *>(&h[4]);
                } else {
                    for (int j = 0; j < 16; ++j) o[j] = __float2bfloat16(v[j]);
                }
            }
        } else {
            for (int j = 0; j < 16; ++j) {
                const int n = nb + j;
                if (n >= N || c0 + j >= NT) break;
                if (Cf) Cf[(size_t)row * ldc + n] = v[j];
                if (Cb) Cb[(size_t)row * ldcb + n] = __float2bfloat16(v[j]);
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(ncols) : "memory");
    if (tid == 0 && s_fail) atomicExch(err, EMPSO_TIMEOUT);
}

cudaError_t gemm(const SurDev &s, cudaStream_t st, int M, int N, int K, const __nv_bfloat16 *A, int lda, int a_mk,
                 const __nv_bfloat16 *B, int ldb, int b_nk, const float *bias, int relu, float *Cf,
                 int ldc, __nv_bfloat16 *Cb, int ldcb)
{
    if (s.tc && s.err && M > 0 && N > 0 && K > 0) {
        const int NT = N >= TNT ? TNT : ((N + 15) / 16) * 16;
        dim3 grid((N + NT - 1) / NT, (M + TM - 1) / TM);
        const size_t smem = (size_t)2 * (TKC / 16) * (TM + NT) * 32;
        const int a_vec = (lda % 8 == 0) && (((size_t)A & 15) == 0);
        const int b_vec = (ldb % 8 == 0) && (((size_t)B & 15) == 0);
        gemm_tc_kernel<<<grid, 128, smem, st>>>(M, N, K, A, lda, a_mk, a_vec, B, ldb, b_nk, b_vec, bias,
                                                relu, Cf, ldc, Cb, ldcb, NT, s.err);
        return cudaGetLastError();
    }
    dim3 grid((N + GBN - 1) / GBN, (M + GBM - 1) / GBM);
    gemm_bf16_kernel<<<grid, 128, 0, st>>>(M, N, K, A, lda, a_mk, B, ldb, b_nk, bias, relu, Cf, ldc,
                                           Cb, ldcb);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// elementwise and reduction kernels
// ---------------------------------------------------------------------------

// x_n = 2 (x - xmin) / (xmax - xmin) - 1, as BF16 rows of the batch
__global__ void normalize_kernel(const float *__restrict__ x, const int *__restrict__ rows, int n,
                                 int K, const double *__restrict__ xmin,
                                 const double *__restrict__ xmax, __nv_bfloat16 *out)
{
    const long long tot = (long long)n * K;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
         e += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(e / K), k = (int)(e % K);
        const int src = rows ? rows[b] : b;
        const float lo = (float)xmin[k], hi = (float)xmax[k];
        out[e] = __float2bfloat16(2.f * (x[(size_t)src * K + k] - lo) / (hi - lo) - 1.f);
    }
}

// y[b] = sum_h relu(Z2[b][h]) w3[h] + b3, one warp per row (fixed order)
__global__ void head_kernel(const float *__restrict__ Z2, int n, int H, const float *__restrict__ w3,
                            const float *__restrict__ b3, float *y)
{
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= n) return;
    float s = 0.f;
    for (int h = lane; h < H; h += 32) s = fmaf(fmaxf(Z2[(size_t)warp * H + h], 0.f), w3[h], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) y[warp] = s + b3[0];
}

// dy = (y - t) / n and the loss 1/(2n) sum (y - t)^2 (one block, fixed order)
__global__ void loss_kernel(const float *__restrict__ y, const float *__restrict__ t, int n,
                            float *dy, float *loss)
{
    __shared__ double red[32];
    double s = 0.0;
    for (int b = threadIdx.x; b < n; b += blockDim.x) {
        const float r = y[b] - t[b];
        dy[b] = r / (float)n;
        s += (double)r * r;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double v = 0.0;
        for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) v += red[w];
        if (loss) *loss = (float)(0.5 * v / n);
    }
}

// dZ2[b][h] = dy[b] w3[h] [Z2 > 0] (FP32 and BF16 copies)
__global__ void dz2_kernel(const float *__restrict__ dy, const float *__restrict__ Z2,
                           const float *__restrict__ w3, int n, int H, float *dZf,
                           __nv_bfloat16 *dZb)
{
    const long long tot = (long long)n * H;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
         e += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(e / H), h = (int)(e % H);
        const float v = Z2[e] > 0.f ? dy[b] * w3[h] : 0.f;
        dZf[e] = v;
        dZb[e] = __float2bfloat16(v);
    }
}

// dZ1 = dA1 [Z1 > 0] (FP32 in place and BF16 copy)
__global__ void relu_back_kernel(float *dA, const float *__restrict__ Z, long long tot,
                                 __nv_bfloat16 *dZb)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
         e += (long long)gridDim.x * blockDim.x) {
        const float v = Z[e] > 0.f ? dA[e] : 0.f;
        dA[e] = v;
        dZb[e] = __float2bfloat16(v);
    }
}

// Column sums g[h] = sum_b v[b][h] over the batch, v = X, or relu(Z) times
// wrow[b]: one CTA of 32 x 32 threads per 32 columns; thread (x, y) sums rows
// y, y + 32, ... of column x, then the 32 partial sums of a column are added
// pairwise in a fixed tree (the same order on every call).
constexpr int CS_T = 32;
__global__ void __launch_bounds__(CS_T * CS_T)
colsum_kernel(const float *__restrict__ X, const float *__restrict__ wrow,
              const float *__restrict__ Zrelu, int n, int H, float *g)
{
    __shared__ float red[CS_T][CS_T + 1];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int h = blockIdx.x * CS_T + tx;
    float s = 0.f;
    if (h < H)
        for (int b = ty; b < n; b += CS_T) {
            float v = X ? X[(size_t)b * H + h] : fmaxf(Zrelu[(size_t)b * H + h], 0.f);
            if (wrow) v *= wrow[b];
            s += v;
        }
    red[ty][tx] = s;
    __syncthreads();
    for (int st = CS_T / 2; st > 0; st >>= 1) {
        if (ty < st) red[ty][tx] += red[ty + st][tx];
        __syncthreads();
    }
    if (ty == 0 && h < H) g[h] = red[0][tx];
}

// out = sum_i v[i]: one CTA, strided partial sums, then a fixed tree
__global__ void sum_kernel(const float *__restrict__ v, int n, float *out)
{
    __shared__ float red[1024];
    float s = 0.f;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += v[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if ((int)threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

// Adam on FP32 master weights, then BF16 copies of the two hidden matrices
__global__ void adam_kernel(float *p, const float *__restrict__ g, float *m, float *v, long long n,
                            float lr, float b1, float b2, float eps, float c1, float c2,
                            __nv_bfloat16 *w1b, long long n_w1, __nv_bfloat16 *w2b, long long off_w2,
                            long long n_w2)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        const float gi = g[e];
        const float mi = b1 * m[e] + (1.f - b1) * gi;
        const float vi = b2 * v[e] + (1.f - b2) * gi * gi;
        m[e] = mi;
        v[e] = vi;
        const float w = p[e] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        p[e] = w;
        if (e < n_w1) w1b[e] = __float2bfloat16(w);
        else if (e >= off_w2 && e < off_w2 + n_w2) w2b[e - off_w2] = __float2bfloat16(w);
    }
}

__global__ void to_bf16_kernel(const float *__restrict__ src, __nv_bfloat16 *dst, long long n)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x)
        dst[e] = __float2bfloat16(src[e]);
}

// Philox4x32-10 (Salmon et al. 2011) for minibatch sampling
__device__ __forceinline__ uint4 philox_s(uint4 c, uint32_t k0, uint32_t k1)
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

// batch rows drawn uniformly from the filled part of the replay buffer (its
// first min(have_host, cap) rows when have_host >= 0, else the device count's);
// with recent > 0 the second half of the batch comes from the newest
// min(recent, filled) pairs instead (the swarm's current neighbourhood)
__global__ void sample_kernel(int *rows, int B, const int *count, int have_host, int cap, uint64_t seed,
                              int step, int recent)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const int total = have_host >= 0 ? have_host : *count;   // pairs appended so far
    const int have = min(total, cap);
    const uint4 w = philox_s(make_uint4((uint32_t)step, (uint32_t)b, 0x5u, 0x7u), (uint32_t)seed,
                             (uint32_t)(seed >> 32));
    if (recent > 0 && b >= B / 2 && have > 0) {
        const int span = min(recent, have);
        const int j = (int)(((unsigned long long)w.x * (unsigned long long)span) >> 32);
        rows[b] = (int)(((long long)total - 1 - j) % cap);
        return;
    }
    rows[b] = have > 0 ? (int)(((unsigned long long)w.x * (unsigned long long)have) >> 32) : 0;
}

// Spearman rank correlation of the k modelled particles' true misfits fk
// and predictions logphi[rows]: ranks by counting (ties by index), one block;
// both keys are staged in shared memory first (k <= 2048)
__global__ void __launch_bounds__(1024)
rank_corr_kernel(const double *__restrict__ fk, const int *__restrict__ rows,
                 const float *__restrict__ logphi, int k, float *rho)
{
    __shared__ double tk[2048];
    __shared__ float pk[2048];
    __shared__ double red[32];
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
        tk[i] = fk[i];
        pk[i] = logphi[rows[i]];
    }
    __syncthreads();
    double d2 = 0.0;
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
        const double ti = tk[i];
        const float pi = pk[i];
        int rt = 0, rp = 0;
        for (int j = 0; j < k; ++j) {
            const double tj = tk[j];
            const float pj = pk[j];
            rt += (tj < ti) || (tj == ti && j < i);
            rp += (pj < pi) || (pj == pi && j < i);
        }
        const double d = (double)(rt - rp);
        d2 += d * d;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) d2 += __shfl_down_sync(0xffffffffu, d2, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = d2;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)blockDim.x / 32; ++w) s += red[w];
        const double kk = (double)k;
        *rho = k > 1 ? (float)(1.0 - 6.0 * s / (kk * (kk * kk - 1.0))) : 1.f;
    }
}

// standardised targets of the batch: (log phi - mu) / sigma
__global__ void targets_kernel(const float *__restrict__ ybuf, const int *__restrict__ rows, int B,
                               const float *__restrict__ stats, float *t)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < B) t[b] = (ybuf[rows[b]] - stats[0]) / stats[1];
}

// mean and standard deviation of the filled replay targets (one block)
__global__ void stats_kernel(const float *__restrict__ ybuf, const int *count, int have_host, int cap,
                             float *stats)
{
    __shared__ double s1[32], s2[32];
    const int n = min(have_host >= 0 ? have_host : *count, cap);
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        a += ybuf[i];
        b += (double)ybuf[i] * ybuf[i];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    if ((threadIdx.x & 31) == 0) {
        s1[threadIdx.x >> 5] = a;
        s2[threadIdx.x >> 5] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double A = 0.0, Bs = 0.0;
        for (int w = 0; w < (int)blockDim.x / 32; ++w) {
            A += s1[w];
            Bs += s2[w];
        }
        double mu = n > 0 ? A / n : 0.0;
        double var = n > 1 ? Bs / n - mu * mu : 1.0;
        stats[0] = (float)mu;
        stats[1] = (float)sqrt(var > 1e-12 ? var : 1e-12);
    }
}

// append (particle, log misfit) pairs; rows with a non-finite misfit are
// skipped.  One block of 1024 threads: the kept rows of each 1024-row chunk
// take consecutive ring slots in row order (an exclusive scan of the keep
// flags), so the buffer order is the same on every run.
__global__ void __launch_bounds__(1024)
append_kernel(const float *__restrict__ x, const double *__restrict__ misfit,
              const int *__restrict__ rows, int n, int K, float *xbuf, float *ybuf, int *count, int cap)
{
    __shared__ int wsum[32];
    __shared__ int slot[1024];
    __shared__ int base, kept;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) base = *count;
    __syncthreads();
    for (int c0 = 0; c0 < n; c0 += 1024) {
        const int m = min(1024, n - c0);
        int ok = 0;
        if (tid < m) {
            const double f = misfit[c0 + tid];
            ok = (isfinite(f) && f > 0.0) ? 1 : 0;
        }
        // inclusive scan within the warp, then over the warp totals
        int v = ok;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += u;
        }
        if (lane == 31) wsum[warp] = v;
        __syncthreads();
        if (warp == 0) {
            int w = wsum[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += u;
            }
            wsum[lane] = w;   // inclusive totals of warps 0..lane
            if (lane == 31) kept = w;
        }
        __syncthreads();
        const int before = v - ok + (warp > 0 ? wsum[warp - 1] : 0);
        slot[tid] = ok ? (base + before) % cap : -1;
        if (tid < m && ok) ybuf[slot[tid]] = (float)log(misfit[c0 + tid]);
        __syncthreads();
        for (int e = tid; e < m * K; e += blockDim.x) {
            const int i = e / K, kk = e % K;
            const int sl = slot[i];
            if (sl < 0) continue;
            const int src = rows ? rows[c0 + i] : c0 + i;
            xbuf[(size_t)sl * K + kk] = x[(size_t)src * K + kk];
        }
        __syncthreads();
        if (tid == 0) base += kept;
        __syncthreads();
    }
    if (tid == 0) *count = base;
}

// predictions back to log-misfit: out = y sigma + mu
__global__ void destandardize_kernel(const float *__restrict__ y, int n, const float *__restrict__ stats,
                                     float *out)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < n) out[b] = y[b] * stats[1] + stats[0];
}

// indices of the k smallest keys (ties to the lower index), one block, P <= 2048
__global__ void __launch_bounds__(1024) select_kernel(const float *__restrict__ key, int P, int k, int *out)
{
    __shared__ float kv[2048];
    __shared__ int iv[2048];
    int N = 1;
    while (N < P) N <<= 1;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        float v = i < P ? key[i] : __int_as_float(0x7f800000);
        if (!(v == v)) v = __int_as_float(0x7f800000);
        kv[i] = v;
        iv[i] = i < P ? i : 0x7fffffff;
    }
    __syncthreads();
    for (int size = 2; size <= N; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = threadIdx.x; t < N / 2; t += blockDim.x) {
                const int lo = 2 * t - (t & (stride - 1)), hi = lo + stride;
                const bool up = (lo & size) == 0;
                const bool lt = kv[hi] < kv[lo] || (kv[hi] == kv[lo] && iv[hi] < iv[lo]);
                const bool gt = kv[lo] < kv[hi] || (kv[lo] == kv[hi] && iv[lo] < iv[hi]);
                if (up ? lt : gt) {
                    const float a = kv[lo];
                    kv[lo] = kv[hi];
                    kv[hi] = a;
                    const int b = iv[lo];
                    iv[lo] = iv[hi];
                    iv[hi] = b;
                }
            }
            __syncthreads();
        }
    for (int i = threadIdx.x; i < k; i += blockDim.x) out[i] = iv[i];
}

// gather selected particles into a compact [k][K] array
__global__ void gather_kernel(const float *__restrict__ x, const int *__restrict__ rows, int k, int K,
                              float *out)
{
    const long long tot = (long long)k * K;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
         e += (long long)gridDim.x * blockDim.x)
        out[e] = x[(size_t)rows[e / K] * K + e % K];
}

// full-swarm fitness (+inf where not modelled) and EM sort keys (modelled:
// true misfit, others: predicted misfit exp(log phi))
__global__ void scatter_kernel(const int *__restrict__ rows, const double *__restrict__ fk, int k,
                               const float *__restrict__ logphi, int P, double *fit, double *rank)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < P) {
        fit[i] = __longlong_as_double(0x7ff0000000000000LL);
        rank[i] = exp((double)logphi[i]);
    }
}

__global__ void scatter_fill_kernel(const int *__restrict__ rows, const double *__restrict__ fk, int k,
                                    double *fit, double *rank)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < k) {
        fit[rows[j]] = fk[j];
        rank[rows[j]] = fk[j];
    }
}

inline int blocks_for(long long n, int per = 256)
{
    long long b = (n + per - 1) / per;
    return (int)(b < 1 ? 1 : (b > 4096 ? 4096 : b));
}

}  // namespace

// ---------------------------------------------------------------------------
// host-side launchers used by api.cu
// ---------------------------------------------------------------------------

// opt the tcgen05 GEMM into its 48 KiB of dynamic shared memory (current device)
cudaError_t sur_prepare_tc()
{
    return cudaFuncSetAttribute(gemm_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
}

cudaError_t sur_forward(const SurDev &s, const __nv_bfloat16 *Xb, int n, float *y, cudaStream_t st)
{
    cudaError_t e;
    if ((e = gemm(s, st, n, s.H, s.K, Xb, s.K, 1, s.W1b, s.K, 1, s.p + s.off_b1, 1, s.Z1, s.H, s.A1b,
                  s.H)))
        return e;
    if ((e = gemm(s, st, n, s.H, s.H, s.A1b, s.H, 1, s.W2b, s.H, 1, s.p + s.off_b2, 0, s.Z2, s.H,
                  nullptr, 0)))
        return e;
    head_kernel<<<(n * 32 + 255) / 256, 256, 0, st>>>(s.Z2, n, s.H, s.p + s.off_w3, s.p + s.off_b3, y);
    return cudaGetLastError();
}

// gradient of the half-MSE on batch (Xb [n][K] BF16, t [n]) into s.g; loss
// to *loss (device float, may be null)
cudaError_t sur_backward(const SurDev &s, const __nv_bfloat16 *Xb, const float *t, int n,
                         float *loss, cudaStream_t st)
{
    cudaError_t e;
    if ((e = sur_forward(s, Xb, n, s.y, st))) return e;
    loss_kernel<<<1, 256, 0, st>>>(s.y, t, n, s.dy, loss);
    // head: g_w3 = sum_b relu(Z2) dy, g_b3 = sum_b dy
    const dim3 cs_grid((s.H + CS_T - 1) / CS_T), cs_block(CS_T, CS_T);
    colsum_kernel<<<cs_grid, cs_block, 0, st>>>(nullptr, s.dy, s.Z2, n, s.H, s.g + s.off_w3);
    sum_kernel<<<1, 1024, 0, st>>>(s.dy, n, s.g + s.off_b3);
    // layer 2
    dz2_kernel<<<blocks_for((long long)n * s.H), 256, 0, st>>>(s.dy, s.Z2, s.p + s.off_w3, n, s.H,
                                                             s.dZf, s.dZb);
    colsum_kernel<<<cs_grid, cs_block, 0, st>>>(s.dZf, nullptr, nullptr, n, s.H, s.g + s.off_b2);
    // g_W2[h][h'] = sum_b dZ2[b][h] A1[b][h']
    if ((e = gemm(s, st, s.H, s.H, n, s.dZb, s.H, 0, s.A1b, s.H, 0, nullptr, 0, s.g + s.off_W2, s.H,
                  nullptr, 0)))
        return e;
    // dA1 = dZ2 W2  -> dZ1 = dA1 [Z1 > 0]
    if ((e = gemm(s, st, n, s.H, s.H, s.dZb, s.H, 1, s.W2b, s.H, 0, nullptr, 0, s.dA, s.H, nullptr, 0)))
        return e;
    relu_back_kernel<<<blocks_for((long long)n * s.H), 256, 0, st>>>(s.dA, s.Z1, (long long)n * s.H,
                                                                     s.dZb);
    colsum_kernel<<<cs_grid, cs_block, 0, st>>>(s.dA, nullptr, nullptr, n, s.H, s.g + s.off_b1);
    // g_W1[h][k] = sum_b dZ1[b][h] X[b][k]
    if ((e = gemm(s, st, s.H, s.K, n, s.dZb, s.H, 0, Xb, s.K, 0, nullptr, 0, s.g + s.off_W1, s.K,
                  nullptr, 0)))
        return e;
    return cudaGetLastError();
}

cudaError_t sur_adam(SurDev &s, cudaStream_t st)
{
    s.t += 1;
    const float c1 = 1.f - powf(s.beta1, (float)s.t), c2 = 1.f - powf(s.beta2, (float)s.t);
    adam_kernel<<<blocks_for(s.n_params), 256, 0, st>>>(s.p, s.g, s.m, s.v, s.n_params, s.lr, s.beta1,
                                                        s.beta2, s.eps, c1, c2, s.W1b,
                                                        (long long)s.H * s.K, s.W2b, s.off_W2,
                                                        (long long)s.H * s.H);
    return cudaGetLastError();
}

cudaError_t sur_refresh_bf16(const SurDev &s, cudaStream_t st)
{
    to_bf16_kernel<<<blocks_for((long long)s.H * s.K), 256, 0, st>>>(s.p + s.off_W1, s.W1b,
                                                                     (long long)s.H * s.K);
    to_bf16_kernel<<<blocks_for((long long)s.H * s.H), 256, 0, st>>>(s.p + s.off_W2, s.W2b,
                                                                     (long long)s.H * s.H);
    return cudaGetLastError();
}

cudaError_t sur_normalize(const SurDev &s, const float *x, const int *rows, int n, __nv_bfloat16 *out,
                          cudaStream_t st)
{
    normalize_kernel<<<blocks_for((long long)n * s.K), 256, 0, st>>>(x, rows, n, s.K, s.xmin, s.xmax,
                                                                     out);
    return cudaGetLastError();
}

cudaError_t sur_predict(const SurDev &s, const float *x, int n, float *logphi, cudaStream_t st)
{
    cudaError_t e;
    if ((e = sur_normalize(s, x, nullptr, n, s.Xb, st))) return e;
    if ((e = sur_forward(s, s.Xb, n, s.y, st))) return e;
    destandardize_kernel<<<(n + 255) / 256, 256, 0, st>>>(s.y, n, s.stats, logphi);
    return cudaGetLastError();
}

cudaError_t sur_append(const SurDev &s, const float *x, const double *misfit, const int *rows, int n,
                       cudaStream_t st)
{
    append_kernel<<<1, 1024, 0, st>>>(x, misfit, rows, n, s.K, s.xbuf, s.ybuf, s.count, s.cap);
    return cudaGetLastError();
}

cudaError_t sur_train(SurDev &s, int steps, int B, cudaStream_t st, int have)
{
    cudaError_t e;
    stats_kernel<<<1, 256, 0, st>>>(s.ybuf, s.count, have, s.cap, s.stats);
    for (int i = 0; i < steps; ++i) {
        sample_kernel<<<(B + 255) / 256, 256, 0, st>>>(s.rows, B, s.count, have, s.cap, s.seed,
                                                       s.sample_step++, s.recent);
        targets_kernel<<<(B + 255) / 256, 256, 0, st>>>(s.ybuf, s.rows, B, s.stats, s.tb);
        // the buffer holds raw positions: scale the batch rows to [-1, 1] in BF16
        if ((e = sur_normalize(s, s.xbuf, s.rows, B, s.Xb, st))) return e;
        if ((e = sur_backward(s, s.Xb, s.tb, B, s.loss, st))) return e;
        if ((e = sur_adam(s, st))) return e;
    }
    return cudaGetLastError();
}

cudaError_t sur_select(const float *key, int P, int k, int *rows, cudaStream_t st)
{
    select_kernel<<<1, 1024, 0, st>>>(key, P, k, rows);
    return cudaGetLastError();
}

cudaError_t sur_rank_corr(const double *fk, const int *rows, const float *logphi, int k, float *rho,
                          cudaStream_t st)
{
    rank_corr_kernel<<<1, 1024, 0, st>>>(fk, rows, logphi, k, rho);
    return cudaGetLastError();
}

cudaError_t sur_gather(const float *x, const int *rows, int k, int K, float *out, cudaStream_t st)
{
    gather_kernel<<<blocks_for((long long)k * K), 256, 0, st>>>(x, rows, k, K, out);
    return cudaGetLastError();
}

cudaError_t sur_scatter(const int *rows, const double *fk, int k, const float *logphi, int P,
                        double *fit, double *rank, cudaStream_t st)
{
    scatter_kernel<<<(P + 255) / 256, 256, 0, st>>>(rows, fk, k, logphi, P, fit, rank);
    scatter_fill_kernel<<<(k + 255) / 256, 256, 0, st>>>(rows, fk, k, fit, rank);
    return cudaGetLastError();
}

}  // namespace empso
