// Allocation-free inverse transform of a k-space state to real space.
//
// Some callers cannot create a context, because creating one allocates
// device memory: applications that reserve their whole device-memory budget
// up front (a fixed pool, or a per-process cap on a shared GPU) and may not
// allocate afterwards, and host frameworks that forbid device allocation in
// the code paths from which they call this library (allocation would
// synchronise the device or fail under their memory policy).  For them this
// file offers pf_state_to_real_noalloc: the same computation as
// pf_set_state_hat + pf_get_state (inverse FFT along z, y, and packed C2R
// along x, in FP64), with every intermediate held in file-scope __device__
// arrays instead of context buffers.  It calls no cudaMalloc/cudaFree and no
// allocating library routine.
#include <cmath>
#include <cstdio>
#include <mutex>
#include <vector>

#include "pf.h"
#include "pf_internal.h"

using namespace pf;

namespace {

// Largest supported problem: nz * ny * (nx/2 + 1) <= kNoallocMaxK complex
// entries per field (64^3 grids: 64 * 64 * 33 = 135168), axes <= 1024.
constexpr long long kNoallocMaxK = 64LL * 64 * 33;
constexpr int kNoallocMaxAxis = 1024;

// Scratch: the partially transformed 4-field state (FP64 complex).  Every
// call overwrites all of the region it later reads, so nothing needs clearing.
static __device__ __align__(256) double2 g_scratch[4 * kNoallocMaxK];
// Per-call tables: twiddles exp(-2 pi i k/n) per axis and wave numbers.
static __device__ __align__(256) double2 g_tw[3][kNoallocMaxAxis];
static __device__ __align__(256) float2 g_tw32[3][kNoallocMaxAxis];
static __device__ __align__(256) double g_k[3][kNoallocMaxAxis];

struct DevPtrs {
    double2* scratch = nullptr;
    double2* tw = nullptr;
    float2* tw32 = nullptr;
    double* k = nullptr;
    bool ready = false;
};

std::mutex g_mu;
std::vector<DevPtrs> g_dev;  // indexed by device ordinal
// errors are reported through pf_last_error(NULL)
int err(int code, const char* msg, cudaError_t e = cudaSuccess) {
    char* dst = create_error_buffer();
    if (e != cudaSuccess)
        std::snprintf(dst, 256, "%s: %s", msg, cudaGetErrorString(e));
    else
        std::snprintf(dst, 256, "%s", msg);
    return code;
}

// One-time set-up per device (with that device current): resolve the device
// addresses of the file-scope arrays.  In host code the array names are only
// host-side stand-ins, so kernels must be given these addresses.
int device_ptrs(int dev, DevPtrs& out) {
    std::lock_guard<std::mutex> lock(g_mu);
    if ((int)g_dev.size() <= dev) g_dev.resize(dev + 1);
    DevPtrs& d = g_dev[dev];
    if (!d.ready) {
        cudaError_t e = cudaGetSymbolAddress((void**)&d.scratch, g_scratch);
        if (e == cudaSuccess) e = cudaGetSymbolAddress((void**)&d.tw, g_tw);
        if (e == cudaSuccess) e = cudaGetSymbolAddress((void**)&d.tw32, g_tw32);
        if (e == cudaSuccess) e = cudaGetSymbolAddress((void**)&d.k, g_k);
        if (e != cudaSuccess) return err(PF_ECUDA, "cudaGetSymbolAddress", e);
        d.ready = true;
    }
    out = d;
    return PF_OK;
}

bool smooth_even_axis(int n) {
    if (n < 4 || n > kNoallocMaxAxis || (n & 1)) return false;
    int m = n;
    for (int p : {2, 3, 5})
        while (m % p == 0) m /= p;
    return m == 1;
}

// Twiddles as the context path builds them: cos and sin of 2 pi k/n in long
// double, the four quarter points exact, rounded to double (and to float).
void twiddles(int n, double2* tw, float2* tw32) {
    for (int k = 0; k < n; ++k) {
        const long double th = 2.0L * 3.141592653589793238462643383279502884L * ((long double)k / (long double)n);
        long double c = cosl(th), s = sinl(th);
        if (4 * k % n == 0) {
            const int q = 4 * k / n;
            c = (q == 0) ? 1.0L : (q == 2 ? -1.0L : 0.0L);
            s = (q == 1) ? 1.0L : (q == 3 ? -1.0L : 0.0L);
        }
        tw[k] = make_double2((double)c, -(double)s);
        tw32[k] = make_float2((float)tw[k].x, (float)tw[k].y);
    }
}

}  // namespace

extern "C" {

int pf_state_to_real_noalloc(const pf_grid* grid, const void* y_hat, double* fields, void* cuda_stream) {
    if (!grid || !y_hat || !fields) return err(PF_EINVAL, "pf_state_to_real_noalloc: NULL argument");
    if (!smooth_even_axis(grid->nx) || !smooth_even_axis(grid->ny) || !smooth_even_axis(grid->nz))
        return err(PF_EUNSUPPORTED, "pf_state_to_real_noalloc: each size must be even, 2,3,5-smooth, 4..1024");
    const long long NK = (long long)grid->nz * grid->ny * (grid->nx / 2 + 1);
    if (NK > kNoallocMaxK)
        return err(PF_EINVAL,
                   "pf_state_to_real_noalloc: grid too large for the static scratch "
                   "(nz*ny*(nx/2+1) must be <= 135168, e.g. 64^3)");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return err(PF_ECUDA, "cudaGetDevice", e);
    DevPtrs d;
    int rc = device_ptrs(dev, d);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)cuda_stream;

    Geo g{};
    g.nx = grid->nx;
    g.ny = grid->ny;
    g.nz = grid->nz;
    g.nxh = g.nx / 2 + 1;
    g.NK = NK;
    g.N = (long long)g.nz * g.ny * g.nx;
    g.invN = 1.0 / (double)g.N;
    g.invN32 = (float)g.invN;
    g.mul_nx = magic_u32((unsigned)g.nx);
    g.mul_nxh = magic_u32((unsigned)g.nxh);
    AxisPlan* plans[3] = {&g.px, &g.py, &g.pz};
    const int ns[3] = {g.nx, g.ny, g.nz};
    const double ds[3] = {grid->dx, grid->dy, grid->dz};
    // host tables for this call, copied into the file-scope device tables
    static thread_local double2 htw[3][kNoallocMaxAxis];
    static thread_local float2 htw32[3][kNoallocMaxAxis];
    static thread_local double hk[3][kNoallocMaxAxis];
    for (int a = 0; a < 3; ++a) {
        if (!make_axis_plan(ns[a], *plans[a]))
            return err(PF_EUNSUPPORTED, "pf_state_to_real_noalloc: cannot factor size");
        twiddles(ns[a], htw[a], htw32[a]);
        const bool half = (a == 0);
        const int len = half ? ns[a] / 2 + 1 : ns[a];
        for (int i = 0; i < len; ++i) {
            int m = i;
            if (!half && i > ns[a] / 2) m = i - ns[a];
            hk[a][i] = 2.0 * 3.14159265358979323846 * m / (ns[a] * ds[a]);
        }
        plans[a]->tw64 = d.tw + a * kNoallocMaxAxis;
        plans[a]->tw32 = d.tw32 + a * kNoallocMaxAxis;
    }
    e = cudaMemcpyToSymbolAsync(g_tw, htw, sizeof htw, 0, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyToSymbolAsync(g_tw32, htw32, sizeof htw32, 0, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyToSymbolAsync(g_k, hk, sizeof hk, 0, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return err(PF_ECUDA, "cudaMemcpyToSymbolAsync", e);
    g.kx = d.k;
    g.ky = d.k + kNoallocMaxAxis;
    g.kz = d.k + 2 * kNoallocMaxAxis;
    Phys ph{};
    StageTerms none{};
    launch_z_stage<double>(g, ph, reinterpret_cast<const double2*>(y_hat), none, nullptr, d.scratch, s);
    launch_y_pass<double>(g, d.scratch, 4, +1, s);
    launch_x_pass<double>(g, ph, XM_C2R_REAL, d.scratch, nullptr, nullptr, nullptr, nullptr, 0, 0, nullptr, fields, s);
    e = cudaGetLastError();
    if (e != cudaSuccess) return err(PF_ECUDA, "kernel launch", e);
    // the host tables above are reused by the next call on this thread
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return err(PF_ECUDA, "cudaStreamSynchronize", e);
    return PF_OK;
}

}  // extern "C"
