// Allocation-free entry point: misfits of gridded velocity models on one grid,
// for callers that cannot allocate device memory (see eval_models_noalloc in
// include/empso.h).  Everything the computation needs beyond the caller's
// inputs and outputs lives in one file-scope device array; host-side
// descriptions (grid, shots, receivers) travel as kernel parameters, so the
// call performs no allocation and no host-to-device copy.  It runs the same
// streaming modelling kernel, field and reduction kernels as eval_models.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>

#include "internal.cuh"

namespace empso {
namespace {

constexpr size_t NOALLOC_SCRATCH_BYTES = 16u << 20;   // 16 MiB per device
constexpr int NOALLOC_MAX_SHOTS = 64;
constexpr int NOALLOC_MAX_RECEIVERS = 1024;
constexpr int NOALLOC_MAX_DEVICES = 64;

// The scratch array: every device that loads the library holds it until the
// process exits.  Host code must never pass its name to a kernel: on the host
// the symbol is only a stand-in, its device address comes from
// cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

std::mutex g_mu;
void *g_scratch_addr[NOALLOC_MAX_DEVICES] = {};

struct SetupParams {
    GridDev g;
    int S, nrec_total, M;
    float sx[NOALLOC_MAX_SHOTS], sz[NOALLOC_MAX_SHOTS], weight[NOALLOC_MAX_SHOTS];
    int rec_begin[NOALLOC_MAX_SHOTS], nrec[NOALLOC_MAX_SHOTS];
    long long doff[NOALLOC_MAX_SHOTS];
    float2 rec[NOALLOC_MAX_RECEIVERS];
};

struct Layout {
    GridDev *grid;
    float *ex, *ez, *wavelet, *Wx, *Wz;
    float2 *rec;
    float *weights;
    Inst *insts;
    double *partial;
    int *counter;
    float *fields;
    float *slots;
    size_t used;
};

size_t up256(size_t b) { return (b + 255) / 256 * 256; }

// Carve the scratch array; `n_slots` wavefield slots follow the fixed part.
Layout carve(unsigned char *base, const GridDev &g, int S, int nrec_total, int M, int n_slots)
{
    Layout L{};
    size_t o = 0;
    auto take = [&](size_t bytes) {
        unsigned char *p = base + o;
        o += up256(bytes);
        return p;
    };
    L.grid = reinterpret_cast<GridDev *>(take(sizeof(GridDev)));
    L.ex = reinterpret_cast<float *>(take(sizeof(float) * g.pitch));
    L.ez = reinterpret_cast<float *>(take(sizeof(float) * g.rows));
    L.wavelet = reinterpret_cast<float *>(take(sizeof(float) * g.nt));
    L.Wx = reinterpret_cast<float *>(take(sizeof(float) * g.nx * g.kx));
    L.Wz = reinterpret_cast<float *>(take(sizeof(float) * g.nz * g.kz));
    L.rec = reinterpret_cast<float2 *>(take(sizeof(float2) * std::max(1, nrec_total)));
    L.weights = reinterpret_cast<float *>(take(sizeof(float) * S));
    L.insts = reinterpret_cast<Inst *>(take(sizeof(Inst) * (size_t)M * S));
    L.partial = reinterpret_cast<double *>(take(sizeof(double) * (size_t)M * S));
    L.counter = reinterpret_cast<int *>(take(sizeof(int)));
    L.fields = reinterpret_cast<float *>(take(sizeof(float) * (size_t)M * g.field));
    L.slots = reinterpret_cast<float *>(take(sizeof(float) * 2 * (size_t)g.field * n_slots));
    L.used = o;
    return L;
}

// Writes the grid descriptor, receiver table, shot weights and instance table
// into the scratch array (one block; everything comes in the parameters).
__global__ void noalloc_setup_kernel(SetupParams p, Layout L, const float *d_obs)
{
    if (threadIdx.x == 0) *L.grid = p.g;
    for (int r = threadIdx.x; r < p.nrec_total; r += blockDim.x) L.rec[r] = p.rec[r];
    for (int s = threadIdx.x; s < p.S; s += blockDim.x) L.weights[s] = p.weight[s];
    for (int q = threadIdx.x; q < p.M * p.S; q += blockDim.x) {
        const int m = q / p.S, s = q % p.S;
        Inst in{};
        in.a = L.fields + (size_t)m * p.g.field;
        in.dobs = d_obs + p.doff[s];
        in.traces = nullptr;
        in.rec = L.rec + p.rec_begin[s];
        in.grid = 0;
        in.nrec = p.nrec[s];
        in.sx = p.sx[s];
        in.sz = p.sz[s];
        in.out = q;
        L.insts[q] = in;
    }
}

empso_status nfail(empso_status s, const std::string &msg)
{
    set_global_error(msg.c_str());
    return s;
}

}  // namespace
}  // namespace empso

using namespace empso;

extern "C" empso_status eval_models_noalloc(const empso_grid *grid, const float *rec_xz,
                                            int32_t nrec_total, const float *vel, int32_t M,
                                            const empso_shot *shots, int32_t S,
                                            const float *d_obs, double *misfit, void *stream)
{
    set_global_error("");
    if (!grid || !shots || S <= 0 || M < 0 || nrec_total < 0 || (nrec_total > 0 && !rec_xz))
        return nfail(EMPSO_INVALID_ARG, "bad grid/shots/receivers");
    if (M > 0 && (!vel || !d_obs || !misfit)) return nfail(EMPSO_INVALID_ARG, "bad vel/d_obs/misfit");
    if (S > NOALLOC_MAX_SHOTS) return nfail(EMPSO_UNSUPPORTED, "more than 64 shots");
    if (nrec_total > NOALLOC_MAX_RECEIVERS) return nfail(EMPSO_UNSUPPORTED, "more than 1024 receivers");
    SetupParams p;
    memset(&p, 0, sizeof p);
    std::string err;
    const empso_status grc = derive_grid(*grid, 0, p.g, err);
    if (grc != EMPSO_OK) return nfail(grc, err);
    const GridDev &g = p.g;
    const float Lx = (grid->nx - 1) * grid->hx, Lz = (grid->nz - 1) * grid->hz;
    long long off = 0;
    for (int s = 0; s < S; ++s) {
        const empso_shot &sh = shots[s];
        if (sh.grid_id != 0 || !(sh.sx >= 0 && sh.sx <= Lx && sh.sz >= 0 && sh.sz <= Lz) ||
            sh.nrec < 0 || sh.rec_begin < 0 || sh.rec_begin + (long long)sh.nrec > nrec_total ||
            !std::isfinite(sh.weight))
            return nfail(EMPSO_INVALID_ARG, "shot " + std::to_string(s) + " out of range");
        for (int r = sh.rec_begin; r < sh.rec_begin + sh.nrec; ++r) {
            const float x = rec_xz[2 * r], z = rec_xz[2 * r + 1];
            if (!(x >= 0 && x <= Lx && z >= 0 && z <= Lz))
                return nfail(EMPSO_INVALID_ARG, "receiver " + std::to_string(r) + " outside the grid");
        }
        p.sx[s] = sh.sx;
        p.sz[s] = sh.sz;
        p.weight[s] = sh.weight;
        p.rec_begin[s] = sh.rec_begin;
        p.nrec[s] = sh.nrec;
        p.doff[s] = off;
        off += (long long)g.nt * sh.nrec;
    }
    for (int r = 0; r < nrec_total; ++r) p.rec[r] = make_float2(rec_xz[2 * r], rec_xz[2 * r + 1]);
    p.S = S;
    p.nrec_total = nrec_total;
    p.M = M;
    if (M == 0) return EMPSO_OK;

    // set-up, once per device: the device address of the scratch array
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NOALLOC_MAX_DEVICES)
        return nfail(EMPSO_CUDA_ERROR, "no current CUDA device");
    unsigned char *base;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_scratch_addr[dev]) {
            void *ptr = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
            if (e != cudaSuccess || !ptr)
                return nfail(EMPSO_CUDA_ERROR, std::string("cudaGetSymbolAddress: ") +
                                                   cudaGetErrorString(e));
            g_scratch_addr[dev] = ptr;
        }
        base = static_cast<unsigned char *>(g_scratch_addr[dev]);
    }

    // size check: the fixed part, the model fields and at least one slot
    const long long n_inst = (long long)M * S;
    const Layout probe = carve(base, g, S, nrec_total, M, 0);
    const size_t slot_bytes = up256(sizeof(float) * 2 * (size_t)g.field);
    if (probe.used + slot_bytes > NOALLOC_SCRATCH_BYTES) {
        char buf[200];
        snprintf(buf, sizeof buf, "needs %zu bytes of scratch for %d model(s) on this grid; the "
                 "allocation-free path has %zu", probe.used + slot_bytes, M, NOALLOC_SCRATCH_BYTES);
        return nfail(EMPSO_UNSUPPORTED, buf);
    }
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return nfail(EMPSO_CUDA_ERROR, "device attribute query failed");
    const int per_sm = std::max(1, wave_max_ctas_per_sm(512));
    long long n_slots = (NOALLOC_SCRATCH_BYTES - probe.used) / slot_bytes;
    n_slots = std::min<long long>({n_slots, n_inst, (long long)sms * per_sm});
    Layout L = carve(base, g, S, nrec_total, M, (int)n_slots);
    p.g.ex = L.ex;
    p.g.ez = L.ez;
    p.g.wavelet = L.wavelet;
    p.g.Wx = L.Wx;
    p.g.Wz = L.Wz;

    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e;
    noalloc_setup_kernel<<<1, 256, 0, st>>>(p, L, d_obs);
    if ((e = cudaGetLastError()) != cudaSuccess ||
        (e = launch_grid_tables(p.g, L.ex, L.ez, L.wavelet, L.Wx, L.Wz, grid->vmax, grid->f0, st)) !=
            cudaSuccess ||
        (e = launch_vel_to_field(p.g, vel, M, L.fields, p.g.field, st)) != cudaSuccess ||
        (e = cudaMemsetAsync(L.counter, 0, sizeof(int), st)) != cudaSuccess ||
        (e = launch_wave(L.grid, L.insts, (int)n_inst, L.counter, L.slots, 2 * p.g.field, (int)n_slots,
                         512, L.partial, st)) != cudaSuccess ||
        (e = launch_finalize(L.partial, L.weights, M, S, misfit, nullptr, st)) != cudaSuccess)
        return nfail(EMPSO_CUDA_ERROR, cudaGetErrorString(e));
    return EMPSO_OK;
}
