// Phase-dependent stiffness: the Hu-Chen fixed-point iterations for
// mechanical equilibrium, Eq. u_gov (Sec. 4.1; Sec. 4.2 names the method).
//
// Local stiffness C(r): the Reuss mix of the cubic matrix and precipitate
// compliances, S(r) = (1 - H) S^m + H S^v with H = sum_v h(phi_v); cubic
// constants (c11, c12, c44) with sigma_xy = 2 c44 eps_xy, compliances
// (s11, s12, s44) with eps_xy = s44 sigma_xy.  Eigenstrain
// eps0 = sum_v h_v eps*_v.  Each iteration solves the homogeneous problem of
// the reference medium C0 with the eigenstress
//   tau = C0:eps0 - (C(r) - C0):(eps_bar + eps(u) - eps0)
// (iteration 0: tau = C0:eps0), in Fourier space
//   eps^(u)_ij = (n_i w_j + n_j w_i)/2,  w = Omega(n) (tau^ n),
//   Omega = (n.C0.n)^-1,
// zero at k = 0 and on the Nyquist planes (no displacement mode there); the
// stress-free mean strain eps_bar solves <C>:eps_bar = <C:(eps0 - eps(u))>.
// The elastic driving force of phi_v is
//   e_v = -sigma:eps*_v - sigma:(S^v - S^m):sigma / 2,
//   sigma = C(r):(eps_bar + eps(u) - eps0).
// Real-space tensor fields are stored as six FP64 components (xx, yy, zz,
// yz, xz, xy; tensor shears) in two four-field groups, k-space ones likewise.
#include <cstdio>

#include "pf_common.cuh"

namespace pf {

namespace {

__device__ __forceinline__ double hval(double f) { return f * f * f * (6.0 * f * f - 15.0 * f + 10.0); }

// sigma = C:e for cubic constants c (Voigt-ordered tensor components)
__device__ __forceinline__ void hooke(const double c[3], const double e[6], double s[6]) {
    const double tr = e[0] + e[1] + e[2];
    s[0] = (c[0] - c[1]) * e[0] + c[1] * tr;
    s[1] = (c[0] - c[1]) * e[1] + c[1] * tr;
    s[2] = (c[0] - c[1]) * e[2] + c[1] * tr;
    s[3] = 2.0 * c[2] * e[3];
    s[4] = 2.0 * c[2] * e[4];
    s[5] = 2.0 * c[2] * e[5];
}

// cubic constants <-> their inverse (the normal block inverts with the same
// functional form; the shear constant maps c44 <-> s44 = 1/(2 c44))
__device__ __host__ __forceinline__ void cubic_inverse(const double a[3], double b[3]) {
    const double d = (a[0] - a[1]) * (a[0] + 2.0 * a[1]);
    b[0] = (a[0] + a[1]) / d;
    b[1] = -a[1] / d;
    b[2] = 1.0 / (2.0 * a[2]);
}

struct PointHC {
    double H, c[3], e0[6];
};

template <typename T>
__device__ __forceinline__ PointHC point_hc(const HCConst& k, const T* __restrict__ R, long long N, long long i) {
    PointHC p;
    double h[3];
    p.H = 0.0;
#pragma unroll
    for (int v = 0; v < 3; ++v) {
        h[v] = hval((double)R[(long long)(1 + v) * N + i]);
        p.H += h[v];
    }
    double s[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) s[a] = (1.0 - p.H) * k.sm[a] + p.H * k.sv[a];
    cubic_inverse(s, p.c);
#pragma unroll
    for (int a = 0; a < 6; ++a) p.e0[a] = h[0] * k.eps[0][a] + h[1] * k.eps[1][a] + h[2] * k.eps[2][a];
    return p;
}

// real slot of component a in the two four-field groups (xx yy zz yz | xz xy)
__device__ __forceinline__ long long slot(int a) { return a; }

template <typename T>
__global__ void k_hc_tau(Geo g, HCConst k, const T* __restrict__ R, const double* __restrict__ eu,
                         const double* __restrict__ ebar, double* __restrict__ tau) {
    const long long N = g.N;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        const PointHC p = point_hc(k, R, N, i);
        double t[6];
        hooke(k.c0, p.e0, t);
        if (eu) {
            double tot[6], cp[3], s[6];
#pragma unroll
            for (int a = 0; a < 6; ++a) tot[a] = ebar[a] + eu[slot(a) * N + i] - p.e0[a];
#pragma unroll
            for (int a = 0; a < 3; ++a) cp[a] = p.c[a] - k.c0[a];
            hooke(cp, tot, s);
#pragma unroll
            for (int a = 0; a < 6; ++a) t[a] -= s[a];
        }
#pragma unroll
        for (int a = 0; a < 6; ++a) tau[slot(a) * N + i] = t[a];
    }
}

// eps^(u) = Gamma(n) : tau^ in place on the six k-space components
__global__ void k_hc_green(Geo g, HCConst k, double2* __restrict__ hk) {
    const long long NK = g.NK;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < NK; r += (long long)gridDim.x * blockDim.x) {
        const int kx = (int)(r % g.nxh);
        const int ky = (int)((r / g.nxh) % g.ny);
        const int kz = (int)(r / ((long long)g.nxh * g.ny));
        const bool nyq = (kx == g.nx / 2) || ((g.ny & 1) == 0 && ky == g.ny / 2) || ((g.nz & 1) == 0 && kz == g.nz / 2);
        const double KX = g.kx[kx], KY = g.ky[ky], KZ = g.kz[kz];
        const double k2 = KX * KX + KY * KY + KZ * KZ;
        if (nyq || k2 == 0.0) {
#pragma unroll
            for (int a = 0; a < 6; ++a) hk[a * NK + r] = make_double2(0.0, 0.0);
            continue;
        }
        const double inv = 1.0 / sqrt(k2);
        const double n[3] = {KX * inv, KY * inv, KZ * inv};
        // acoustic tensor of C0 along n and its inverse by cofactors
        const double c11 = k.c0[0], c12 = k.c0[1], c44 = k.c0[2];
        const double a = c44 + (c11 - c44) * n[0] * n[0], b = c44 + (c11 - c44) * n[1] * n[1];
        const double c = c44 + (c11 - c44) * n[2] * n[2];
        const double d = (c12 + c44) * n[0] * n[1], e = (c12 + c44) * n[0] * n[2], f = (c12 + c44) * n[1] * n[2];
        const double A11 = b * c - f * f, A12 = e * f - d * c, A13 = d * f - b * e;
        const double A22 = a * c - e * e, A23 = d * e - a * f, A33 = a * b - d * d;
        const double idet = 1.0 / (a * A11 + d * A12 + e * A13);
        double2 t[6];
#pragma unroll
        for (int q = 0; q < 6; ++q) t[q] = hk[q * NK + r];
        // tau^ n (tau symmetric: xx yy zz yz xz xy)
        const double2 tn0 = {t[0].x * n[0] + t[5].x * n[1] + t[4].x * n[2], t[0].y * n[0] + t[5].y * n[1] + t[4].y * n[2]};
        const double2 tn1 = {t[5].x * n[0] + t[1].x * n[1] + t[3].x * n[2], t[5].y * n[0] + t[1].y * n[1] + t[3].y * n[2]};
        const double2 tn2 = {t[4].x * n[0] + t[3].x * n[1] + t[2].x * n[2], t[4].y * n[0] + t[3].y * n[1] + t[2].y * n[2]};
        double2 w[3];
        w[0] = {(A11 * tn0.x + A12 * tn1.x + A13 * tn2.x) * idet, (A11 * tn0.y + A12 * tn1.y + A13 * tn2.y) * idet};
        w[1] = {(A12 * tn0.x + A22 * tn1.x + A23 * tn2.x) * idet, (A12 * tn0.y + A22 * tn1.y + A23 * tn2.y) * idet};
        w[2] = {(A13 * tn0.x + A23 * tn1.x + A33 * tn2.x) * idet, (A13 * tn0.y + A23 * tn1.y + A33 * tn2.y) * idet};
        const int I[6] = {0, 1, 2, 1, 0, 0}, J[6] = {0, 1, 2, 2, 2, 1};
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            const int i = I[q], j = J[q];
            hk[q * NK + r] = make_double2(0.5 * (n[i] * w[j].x + n[j] * w[i].x), 0.5 * (n[i] * w[j].y + n[j] * w[i].y));
        }
    }
}

// per-block partials: [0..2] sums of c11, c12, c44; [3..8] sums of
// C:(eps0 - eps(u)); [9] max |eps(u) - eps(u)_prev|; [10] max |eps0|
template <typename T>
__global__ void __launch_bounds__(256) k_hc_stats(Geo g, HCConst k, const T* __restrict__ R,
                                                  const double* __restrict__ eu, const double* __restrict__ eu_prev,
                                                  double* __restrict__ part) {
    const long long N = g.N;
    double acc[11];
#pragma unroll
    for (int q = 0; q < 11; ++q) acc[q] = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        const PointHC p = point_hc(k, R, N, i);
        double d[6], s[6];
#pragma unroll
        for (int a = 0; a < 6; ++a) d[a] = p.e0[a] - eu[slot(a) * N + i];
        hooke(p.c, d, s);
#pragma unroll
        for (int a = 0; a < 3; ++a) acc[a] += p.c[a];
#pragma unroll
        for (int a = 0; a < 6; ++a) acc[3 + a] += s[a];
        if (eu_prev) {
#pragma unroll
            for (int a = 0; a < 6; ++a) acc[9] = fmax(acc[9], fabs(eu[slot(a) * N + i] - eu_prev[slot(a) * N + i]));
        }
#pragma unroll
        for (int a = 0; a < 6; ++a) acc[10] = fmax(acc[10], fabs(p.e0[a]));
    }
    __shared__ double red[11][8];
#pragma unroll
    for (int q = 0; q < 11; ++q) {
        double v = acc[q];
        for (int o = 16; o > 0; o >>= 1) {
            const double w = __shfl_xor_sync(0xffffffffu, v, o);
            v = q < 9 ? v + w : fmax(v, w);
        }
        if ((threadIdx.x & 31) == 0) red[q][threadIdx.x >> 5] = v;
    }
    __syncthreads();
    if (threadIdx.x < 11) {
        const int q = threadIdx.x;
        double v = red[q][0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) v = q < 9 ? v + red[q][w] : fmax(v, red[q][w]);
        part[(long long)blockIdx.x * 11 + q] = v;
    }
}

// e_v = -sigma:eps*_v - sigma:dS:sigma / 2 into E [3][N] (compute type)
template <typename T>
__global__ void k_hc_force(Geo g, HCConst k, const T* __restrict__ R, const double* __restrict__ eu,
                           const double* __restrict__ ebar, T* __restrict__ E) {
    const long long N = g.N;
    const double ds[3] = {k.sv[0] - k.sm[0], k.sv[1] - k.sm[1], k.sv[2] - k.sm[2]};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        const PointHC p = point_hc(k, R, N, i);
        double el[6], s[6];
#pragma unroll
        for (int a = 0; a < 6; ++a) el[a] = ebar[a] + eu[slot(a) * N + i] - p.e0[a];
        hooke(p.c, el, s);
        const double sdS = ds[0] * (s[0] * s[0] + s[1] * s[1] + s[2] * s[2]) +
                           2.0 * ds[1] * (s[0] * s[1] + s[1] * s[2] + s[0] * s[2]) +
                           2.0 * ds[2] * (s[3] * s[3] + s[4] * s[4] + s[5] * s[5]);
#pragma unroll
        for (int v = 0; v < 3; ++v) {
            const double* ev = k.eps[v];
            const double se = s[0] * ev[0] + s[1] * ev[1] + s[2] * ev[2] + 2.0 * (s[3] * ev[3] + s[4] * ev[4] + s[5] * ev[5]);
            E[(long long)v * N + i] = (T)(-se - 0.5 * sdS);
        }
    }
}

// sum over points of sigma:eps_el / 2 (the elastic energy density), per block
template <typename T>
__global__ void __launch_bounds__(256) k_hc_energy(Geo g, HCConst k, const T* __restrict__ R,
                                                   const double* __restrict__ eu, const double* __restrict__ ebar,
                                                   double* __restrict__ part) {
    const long long N = g.N;
    double acc = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        const PointHC p = point_hc(k, R, N, i);
        double el[6], s[6];
#pragma unroll
        for (int a = 0; a < 6; ++a) el[a] = ebar[a] + eu[slot(a) * N + i] - p.e0[a];
        hooke(p.c, el, s);
        acc += 0.5 * (s[0] * el[0] + s[1] * el[1] + s[2] * el[2] + 2.0 * (s[3] * el[3] + s[4] * el[4] + s[5] * el[5]));
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    __shared__ double red[8];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double v = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[w];
        part[blockIdx.x] = v;
    }
}

}  // namespace

int hc_blocks() { return 152 * 8; }

void hc_constants(double C11, double C12, double C44, double C11v, double C12v, double C44v,
                  const double eps[3][6], HCConst& k) {
    const double cm[3] = {C11, C12, C44}, cv[3] = {C11v, C12v, C44v};
    cubic_inverse(cm, k.sm);
    cubic_inverse(cv, k.sv);
    for (int a = 0; a < 3; ++a) k.c0[a] = 0.5 * (cm[a] + cv[a]);
    for (int v = 0; v < 3; ++v)
        for (int a = 0; a < 6; ++a) k.eps[v][a] = eps[v][a];
}

template <typename T>
void launch_hc_tau(const Geo& g, const HCConst& k, const void* R, const double* eu, const double* ebar, double* tau,
                   cudaStream_t s) {
    k_hc_tau<T><<<hc_blocks(), 256, 0, s>>>(g, k, reinterpret_cast<const T*>(R), eu, ebar, tau);
}
void launch_hc_green(const Geo& g, const HCConst& k, double2* hk, cudaStream_t s) {
    k_hc_green<<<hc_blocks(), 256, 0, s>>>(g, k, hk);
}
template <typename T>
void launch_hc_stats(const Geo& g, const HCConst& k, const void* R, const double* eu, const double* eu_prev,
                     double* part, cudaStream_t s) {
    k_hc_stats<T><<<hc_blocks(), 256, 0, s>>>(g, k, reinterpret_cast<const T*>(R), eu, eu_prev, part);
}
template <typename T>
void launch_hc_force(const Geo& g, const HCConst& k, const void* R, const double* eu, const double* ebar, void* E,
                     cudaStream_t s) {
    k_hc_force<T><<<hc_blocks(), 256, 0, s>>>(g, k, reinterpret_cast<const T*>(R), eu, ebar, reinterpret_cast<T*>(E));
}
template <typename T>
void launch_hc_energy(const Geo& g, const HCConst& k, const void* R, const double* eu, const double* ebar,
                      double* part, cudaStream_t s) {
    k_hc_energy<T><<<hc_blocks(), 256, 0, s>>>(g, k, reinterpret_cast<const T*>(R), eu, ebar, part);
}

template void launch_hc_tau<float>(const Geo&, const HCConst&, const void*, const double*, const double*, double*,
                                   cudaStream_t);
template void launch_hc_tau<double>(const Geo&, const HCConst&, const void*, const double*, const double*, double*,
                                    cudaStream_t);
template void launch_hc_stats<float>(const Geo&, const HCConst&, const void*, const double*, const double*, double*,
                                     cudaStream_t);
template void launch_hc_stats<double>(const Geo&, const HCConst&, const void*, const double*, const double*, double*,
                                      cudaStream_t);
template void launch_hc_force<float>(const Geo&, const HCConst&, const void*, const double*, const double*, void*,
                                     cudaStream_t);
template void launch_hc_force<double>(const Geo&, const HCConst&, const void*, const double*, const double*, void*,
                                      cudaStream_t);
template void launch_hc_energy<float>(const Geo&, const HCConst&, const void*, const double*, const double*, double*,
                                      cudaStream_t);
template void launch_hc_energy<double>(const Geo&, const HCConst&, const void*, const double*, const double*, double*,
                                       cudaStream_t);

}  // namespace pf
