// Observed-data preprocessing (section "Testing approach": the recorded data
// are low-pass filtered below the modelling band before the inversion):
// band-limited resampling of traces with the Blackman-windowed sinc
//   h(tau) = 2 fc sinc(2 fc tau) w(tau / W),
//   w(u) = 0.42 + 0.5 cos(pi u) + 0.08 cos(2 pi u) for |u| < 1, else 0,
//   out[s][m][r] = dt_in sum_n in[s][n][r] h(m dt_out - n dt_in),
// records starting at t = 0 and zero outside them.  With dt_out = dt_in it is
// a zero-phase low-pass.
//
// One block per (shot, tile of MT consecutive output times).  The taps of the
// tile's input window are computed once into shared memory, k-major
// (taps[k][j], j = output time in the tile), so one input sample meets its MT
// taps in two 16-byte shared loads.  Each thread accumulates the MT outputs of
// one receiver, reading each input sample of the window once (coalesced across
// receivers).
#include "internal.cuh"

namespace empso {

namespace {

constexpr int MT = 8;

__device__ __forceinline__ float bsinc_tap(double tau, double fc, double W, double dt_in)
{
    const double u = tau / W;
    if (u <= -1.0 || u >= 1.0) return 0.f;
    const float uf = (float)u;
    const float w = 0.42f + 0.5f * cospif(uf) + 0.08f * cospif(2.f * uf);
    const float x = (float)(2.0 * fc * tau);
    const float sinc = (x == 0.f) ? 1.f : sinpif(x) / (3.14159265358979f * x);
    return (float)(dt_in * 2.0 * fc) * sinc * w;
}

__global__ void __launch_bounds__(256)
lowpass_kernel(const float *__restrict__ in, int nt_in, int nrec, double dt_in,
               float *__restrict__ out, int nt_out, double dt_out, double fc, double W)
{
    extern __shared__ __align__(16) float taps[];   // [span][MT]
    const int s = blockIdx.y, m0 = blockIdx.x * MT;
    const int mcount = min(MT, nt_out - m0);
    const double t0 = m0 * dt_out, t1 = (m0 + mcount - 1) * dt_out;
    const int n_lo = max((int)ceil((t0 - W) / dt_in), 0);
    const int n_hi = min((int)floor((t1 + W) / dt_in), nt_in - 1);
    const int span = n_hi >= n_lo ? n_hi - n_lo + 1 : 0;
    for (int e = threadIdx.x; e < span * MT; e += blockDim.x) {
        const int k = e / MT, j = e % MT;
        taps[e] = j < mcount ? bsinc_tap((m0 + j) * dt_out - (double)(n_lo + k) * dt_in, fc, W, dt_in)
                             : 0.f;
    }
    __syncthreads();
    const float4 *t4 = reinterpret_cast<const float4 *>(taps);
    for (int r = threadIdx.x; r < nrec; r += blockDim.x) {
        float acc[MT];
#pragma unroll
        for (int j = 0; j < MT; ++j) acc[j] = 0.f;
        const float *x = in + ((size_t)s * nt_in + n_lo) * nrec + r;
        for (int k = 0; k < span; ++k) {
            const float xv = __ldg(x + (size_t)k * nrec);
            const float4 a = t4[2 * k], b = t4[2 * k + 1];
            acc[0] = fmaf(a.x, xv, acc[0]);
            acc[1] = fmaf(a.y, xv, acc[1]);
            acc[2] = fmaf(a.z, xv, acc[2]);
            acc[3] = fmaf(a.w, xv, acc[3]);
            acc[4] = fmaf(b.x, xv, acc[4]);
            acc[5] = fmaf(b.y, xv, acc[5]);
            acc[6] = fmaf(b.z, xv, acc[6]);
            acc[7] = fmaf(b.w, xv, acc[7]);
        }
#pragma unroll
        for (int j = 0; j < MT; ++j)
            if (j < mcount) out[((size_t)s * nt_out + m0 + j) * nrec + r] = acc[j];
    }
}

}  // namespace

// largest input window of one tile (taps per output time x MT floats of
// shared memory)
long long lowpass_span(double dt_in, double dt_out, double W)
{
    return (long long)std::ceil(((MT - 1) * dt_out + 2.0 * W) / dt_in) + 2;
}

size_t lowpass_smem_bytes(long long span) { return sizeof(float) * MT * (size_t)span; }

cudaError_t lowpass_configure(size_t smem)
{
    return cudaFuncSetAttribute(lowpass_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

cudaError_t launch_lowpass(const float *in, int S, int nt_in, int nrec, double dt_in, float *out,
                           int nt_out, double dt_out, double fc, double W, size_t smem,
                           cudaStream_t st)
{
    const int threads = nrec >= 256 ? 256 : ((nrec + 31) / 32) * 32;
    dim3 grid((nt_out + MT - 1) / MT, S);
    lowpass_kernel<<<grid, threads, smem, st>>>(in, nt_in, nrec, dt_in, out, nt_out, dt_out, fc, W);
    return cudaGetLastError();
}

}  // namespace empso
