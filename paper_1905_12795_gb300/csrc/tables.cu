// Per-grid tables and the two-grid parameterisation (section "Testing
// approach": control nodes interpolated onto the FD grid; JSON nbpml damping
// layer; Ricker source wavelet).
#include "internal.cuh"

namespace empso {

// Damping: eta(d) = eta_max (d / L)^2 for a node d metres into the layer
// (measured from its inner edge), L = pad h, eta_max = 3 vmax ln(1/R) / (2 L),
// R = 1e-3 (Collino & Tsogka 2001).  Stored pre-multiplied by dt / 2 per
// buffer column (x) and buffer row (z); halo cells get 0.
__device__ double damping_eta(int I, int n, int pad, double h, double vmax)
{
    if (pad <= 0) return 0.0;
    double d = 0.0;
    if (I < pad) d = (double)(pad - I) * h;
    else if (I > pad + n - 1) d = (double)(I - (pad + n - 1)) * h;
    if (d <= 0.0) return 0.0;
    double L = pad * h;
    double etamax = 3.0 * vmax * log(1000.0) / (2.0 * L);
    double q = d / L;
    return etamax * q * q;
}

__global__ void damping_kernel(GridDev g, float *ex, float *ez, double vmax)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < g.pitch) {
        int I = t - HALO;
        float v = 0.f;
        if (I >= 0 && I < g.NX) v = (float)(damping_eta(I, g.nx, g.pad, g.hx, vmax) * g.dt * 0.5);
        ex[t] = v;
    }
    if (t < g.rows) {
        int J = t - HALO;
        float v = 0.f;
        if (J >= 0 && J < g.NZ) v = (float)(damping_eta(J, g.nz, g.pad, g.hz, vmax) * g.dt * 0.5);
        ez[t] = v;
    }
}

// Ricker wavelet r(t) = (1 - 2 a) e^{-a}, a = (pi f0 (t - 1/f0))^2, sampled at
// t_n = n dt.
__global__ void wavelet_kernel(float *w, int nt, double dt, double f0)
{
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= nt) return;
    double tau = n * dt - 1.0 / f0;
    double a = 3.14159265358979323846 * f0 * tau;
    a = a * a;
    w[n] = (float)((1.0 - 2.0 * a) * exp(-a));
}

// Interpolation weights of K uniformly spaced control nodes (node k at grid
// index k (n-1)/(K-1)) onto the n grid nodes: column k is the interpolant of
// the k-th unit vector.  Mode 0: natural cubic spline (second derivatives
// solved by the Thomas algorithm on the tridiagonal system
// M_{j-1} + 4 M_j + M_{j+1} = 6 (y_{j+1} - 2 y_j + y_{j-1}) / H^2,
// M_0 = M_{K-1} = 0).  Mode 1: piecewise linear.  One block per k.
__global__ void interp_weights_kernel(float *W, int K, int n, int mode)
{
    __shared__ double M[64];
    __shared__ double cp[64];
    __shared__ double dp[64];
    const int k = blockIdx.x;
    const double H = (double)(n - 1) / (double)(K - 1);
    if (threadIdx.x == 0) {
        for (int j = 0; j < K; ++j) M[j] = 0.0;
        if (mode == 0 && K > 2) {
            // unknowns M_1 .. M_{K-2}; forward sweep
            int m = K - 2;
            for (int r = 0; r < m; ++r) {
                int j = r + 1;
                double rhs = 6.0 * (((j + 1) == k) - 2.0 * (j == k) + ((j - 1) == k)) / (H * H);
                double b = 4.0, a = (r > 0) ? 1.0 : 0.0, c = 1.0;
                double den = b - a * (r > 0 ? cp[r - 1] : 0.0);
                cp[r] = c / den;
                dp[r] = (rhs - a * (r > 0 ? dp[r - 1] : 0.0)) / den;
            }
            for (int r = m - 1; r >= 0; --r)
                M[r + 1] = dp[r] - (r < m - 1 ? cp[r] * M[r + 2] : 0.0);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double xi = (double)i;
        int seg = (int)floor(xi / H);
        seg = seg > K - 2 ? K - 2 : (seg < 0 ? 0 : seg);
        double t = (xi - seg * H) / H;
        double y0 = (seg == k) ? 1.0 : 0.0;
        double y1 = (seg + 1 == k) ? 1.0 : 0.0;
        double s = (1.0 - t) * y0 + t * y1;
        if (mode == 0) {
            double u = 1.0 - t;
            s += H * H / 6.0 * ((u * u * u - u) * M[seg] + (t * t * t - t) * M[seg + 1]);
        }
        W[(size_t)i * K + k] = (float)s;
    }
}

cudaError_t launch_grid_tables(const GridDev &g, float *ex, float *ez, float *wavelet,
                               float *Wx, float *Wz, double vmax_damp, double f0,
                               cudaStream_t st)
{
    int n = g.pitch > g.rows ? g.pitch : g.rows;
    damping_kernel<<<(n + 255) / 256, 256, 0, st>>>(g, ex, ez, vmax_damp);
    wavelet_kernel<<<(g.nt + 255) / 256, 256, 0, st>>>(wavelet, g.nt, (double)g.dt, f0);
    interp_weights_kernel<<<g.kx, 256, 0, st>>>(Wx, g.kx, g.nx, g.mode);
    interp_weights_kernel<<<g.kz, 256, 0, st>>>(Wz, g.kz, g.nz, g.mode);
    return cudaGetLastError();
}

// Taps of the irregular level-wise control grid ("Testing approach": a
// variable node spacing, nodes bilinearly interpolated to the FD grid).
// Level l lies at depth level_z[l] and holds the nodes level_off[l] ..
// level_off[l+1]-1 at increasing x positions node_x[..].  For physical node
// (i, j) at (x, z) = (i hx, j hz): the two levels bracketing z (the first or
// last level alone above/below them) with weight 1 - b and b, and on each
// level the two nodes bracketing x (the end node alone beyond the ends) with
// weight 1 - a and a.  One thread per point, positions in FP64.
__global__ void level_taps_kernel(int nx, int nz, double hx, double hz, int L,
                                  const float *__restrict__ level_z, const int *__restrict__ level_off,
                                  const float *__restrict__ node_x, int4 *lidx, float4 *lw)
{
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= (long long)nx * nz) return;
    const int i = (int)(e % nx), j = (int)(e / nx);
    const double x = i * hx, z = j * hz;
    int la, lb;
    double b = 0.0;
    if (z <= (double)level_z[0]) {
        la = lb = 0;
    } else if (z >= (double)level_z[L - 1]) {
        la = lb = L - 1;
    } else {
        la = 0;
        while (!(z < (double)level_z[la + 1])) ++la;
        lb = la + 1;
        b = (z - level_z[la]) / ((double)level_z[lb] - (double)level_z[la]);
    }
    int n0[2], n1[2];
    double a[2];
    const int lv[2] = {la, lb};
    for (int s = 0; s < 2; ++s) {
        const int o = level_off[lv[s]], n = level_off[lv[s] + 1] - o;
        const float *xs = node_x + o;
        if (n == 1 || x <= (double)xs[0]) {
            n0[s] = n1[s] = o;
            a[s] = 0.0;
        } else if (x >= (double)xs[n - 1]) {
            n0[s] = n1[s] = o + n - 1;
            a[s] = 0.0;
        } else {
            int k = 0;
            while (!(x < (double)xs[k + 1])) ++k;
            n0[s] = o + k;
            n1[s] = o + k + 1;
            a[s] = (x - xs[k]) / ((double)xs[k + 1] - (double)xs[k]);
        }
    }
    lidx[e] = make_int4(n0[0], n1[0], n0[1], n1[1]);
    lw[e] = make_float4((float)((1.0 - b) * (1.0 - a[0])), (float)((1.0 - b) * a[0]),
                        (float)(b * (1.0 - a[1])), (float)(b * a[1]));
}

cudaError_t launch_level_taps(const GridDev &g, int L, const float *level_z, const int *level_off,
                              const float *node_x, int4 *lidx, float4 *lw, cudaStream_t st)
{
    const long long n = (long long)g.nx * g.nz;
    level_taps_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(g.nx, g.nz, g.hx, g.hz, L, level_z,
                                                                  level_off, node_x, lidx, lw);
    return cudaGetLastError();
}

// Model field a = v^2 dt^2 in buffer layout from the control nodes of one
// particle per blockIdx.y: v(i, j) = sum_kz Wz[j][kz] sum_kx C[kz][kx] Wx[i][kx],
// clipped to [vmin, vmax], edge-extended into the damping pad; 0 in the halo
// and in the alignment columns past NX.  Optionally also writes the physical
// model [nz][nx] (m/s).
__global__ void interp_kernel(GridDev g, const float *__restrict__ particles, float *a_fields,
                              long long field_stride, float *vel_out, int col_blocks)
{
    extern __shared__ float C[];
    const int p = blockIdx.y;
    const int K = g.K;
    for (int k = threadIdx.x; k < K; k += blockDim.x) C[k] = particles[(size_t)p * K + k];
    __syncthreads();
    // one buffer column per thread, a strided set of its rows per CTA
    const int c = (blockIdx.x % col_blocks) * blockDim.x + threadIdx.x;
    if (c >= g.pitch) return;
    const int row_blocks = gridDim.x / col_blocks;
    const int rows = (int)(g.field / g.pitch);
    float *a = a_fields + p * field_stride;
    const int I = c - HALO;
    const bool col_in = I >= 0 && I < g.NX;
    const int i = min(max(I - g.pad, 0), g.nx - 1);
    const float *wx = g.Wx + (size_t)i * g.kx;
    // the column's x-sums t_kz = sum_kx C[kz][kx] Wx[i][kx] are the same for
    // every row: with up to KZ_REG rows of nodes they are formed once, in
    // registers, and each point takes only its kz-sum (the same operations in
    // the same order as forming them per point)
    constexpr int KZ_REG = 16;
    const bool reg = g.mode != 2 && g.kz <= KZ_REG;
    float T[KZ_REG];
#pragma unroll
    for (int kz = 0; kz < KZ_REG; ++kz) {
        float t = 0.f;
        if (reg && col_in && kz < g.kz)
            for (int kx = 0; kx < g.kx; ++kx) t = fmaf(C[kz * g.kx + kx], wx[kx], t);
        T[kz] = t;
    }
    for (int r = blockIdx.x / col_blocks; r < rows; r += row_blocks) {
        const int J = r - HALO;
        float out = 0.f;
        if (col_in && J >= 0 && J < g.NZ) {
            const int j = min(max(J - g.pad, 0), g.nz - 1);
            float v = 0.f;
            if (reg) {
                const float *wz = g.Wz + (size_t)j * g.kz;
#pragma unroll
                for (int kz = 0; kz < KZ_REG; ++kz)
                    if (kz < g.kz) v = fmaf(__ldg(wz + kz), T[kz], v);
            } else if (g.mode == 2) {
                const int4 q = g.lidx[(size_t)j * g.nx + i];
                const float4 w = g.lw[(size_t)j * g.nx + i];
                v = fmaf(w.x, C[q.x], fmaf(w.y, C[q.y], fmaf(w.z, C[q.z], w.w * C[q.w])));
            } else {
                const float *wz = g.Wz + (size_t)j * g.kz;
                for (int kz = 0; kz < g.kz; ++kz) {
                    float t = 0.f;
                    for (int kx = 0; kx < g.kx; ++kx) t = fmaf(C[kz * g.kx + kx], wx[kx], t);
                    v = fmaf(wz[kz], t, v);
                }
            }
            if (g.water_z > 0.f && (double)j * g.hz <= (double)g.water_z) v = g.v_water;
            v = fminf(fmaxf(v, g.vmin), g.vmax);
            float vd = v * g.dt;
            out = vd * vd;
            if (vel_out && I - g.pad == i && J - g.pad == j)
                vel_out[(size_t)p * g.nx * g.nz + (size_t)j * g.nx + i] = v;
        }
        a[(size_t)r * g.pitch + c] = out;
    }
}

cudaError_t launch_interp(const GridDev &g, const float *particles, int P, float *a_fields,
                          long long field_stride, float *vel_out, cudaStream_t st)
{
    if (P <= 0) return cudaSuccess;
    const int K = g.K;
    const int T = 128;
    const int col_blocks = (g.pitch + T - 1) / T;
    const int rows = (int)(g.field / g.pitch);
    // about 16 rows per thread, at least 2048 CTAs over the batch when the rows allow
    int row_blocks = std::max((rows + 15) / 16, (2048 + P * col_blocks - 1) / (P * col_blocks));
    row_blocks = std::min(row_blocks, rows);
    dim3 grid(col_blocks * row_blocks, P);
    interp_kernel<<<grid, T, K * sizeof(float), st>>>(g, particles, a_fields, field_stride, vel_out,
                                                       col_blocks);
    return cudaGetLastError();
}

// Model field from a gridded physical model [nz][nx] (m/s), edge-extended
// into the pad.
__global__ void vel_field_kernel(GridDev g, const float *__restrict__ vel, float *a_fields,
                                 long long field_stride)
{
    const int m = blockIdx.y;
    float *a = a_fields + m * field_stride;
    const float *v0 = vel + (size_t)m * g.nx * g.nz;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < g.field;
         e += (long long)gridDim.x * blockDim.x) {
        int r = (int)(e / g.pitch), c = (int)(e % g.pitch);
        int I = c - HALO, J = r - HALO;
        float out = 0.f;
        if (I >= 0 && I < g.NX && J >= 0 && J < g.NZ) {
            int i = min(max(I - g.pad, 0), g.nx - 1);
            int j = min(max(J - g.pad, 0), g.nz - 1);
            float vd = v0[(size_t)j * g.nx + i] * g.dt;
            out = vd * vd;
        }
        a[e] = out;
    }
}

cudaError_t launch_vel_to_field(const GridDev &g, const float *vel, int M, float *a_fields,
                                long long field_stride, cudaStream_t st)
{
    if (M <= 0) return cudaSuccess;
    int blocks = (int)((g.field + 255) / 256);
    if (blocks > 1024) blocks = 1024;
    dim3 grid(blocks, M);
    vel_field_kernel<<<grid, 256, 0, st>>>(g, vel, a_fields, field_stride);
    return cudaGetLastError();
}

}  // namespace empso
