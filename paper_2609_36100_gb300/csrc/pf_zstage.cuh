// Pass kernels of the pseudospectral ImEx-ARK right-hand side (Sec. 4.2/4.4
// of the paper) on sm_103a.
//
// One explicit right-hand-side evaluation f^E(z) is nine memory passes over
// field-major arrays ([field][z][y][x] real, [field][kz][ky][kx] half
// spectrum), each one shared-memory FFT along one axis with the pointwise
// work of that point of the method fused into it:
//   z: stage assembly + diagonal implicit solve (Eq. ARK_stage) + inverse FFT
//   y: inverse FFT
//   x: C2R -> real X, phi_v; h(phi_v) -> R2C (or the whole RHS when the
//      eigenstrains vanish)
//   y: forward FFT of h          z: forward FFT, Green's contraction
//   y: inverse FFT of e          B_vq(k/|k|) h^_q, inverse FFT
//   x: C2R of e, KKS mu, g_v, q -> R2C        y: forward FFT
//   z: forward FFT + k-space scaling -> f^E (-M k^2, -L)
// Step completion (Eq. ARK_method), the embedded local error (Eq.
// ARK_embedding) and its WRMS norm (Eqs. wrms_norm, wrms_weights) are three
// more passes; this file holds the two that combine stages (stage assembly
// and step completion) with the transform fused in, for the FP64 form; the
// FP32-bulk form runs the same combinations as streams (k_stage_assemble_df,
// k_step_complete_df) followed by an in-place inverse z pass, which keeps the
// memory stream and the transform apart.  The state is always FP64, the stage
// vectors FP64 or, in the FP32-bulk form, double-float.
#pragma once
#include "pf_common.cuh"

namespace pf {
// ---------------------------------------------------------------------------
// z pass: stage assembly + implicit solve + inverse FFT along z
//   r = y + sum_j (dt A^I_ij) lambda z_j + (dt A^E_ij) f^E_j
//   z_i = r / (1 - dt A^I_ii lambda)
// The tile is assembled in shared memory before the transform (every load of
// an element issued together); each element is formed once.
// ---------------------------------------------------------------------------
template <typename T, int TX, bool R16, int PID, int MAXT>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? 3 : 2) k_z_stage(Geo g, Phys ph, const double2* __restrict__ y, StageTerms st,
                                                      double2* __restrict__ zout,
                                                      typename Cx<T>::t* __restrict__ W) {
    PF_SKIP_INACTIVE(g);
    if (y_swapped(g)) y = g.yother;
    using T2 = typename Cx<T>::t;
    extern __shared__ __align__(16) unsigned char smraw[];
    T2* A = reinterpret_cast<T2*>(smraw);
    T2* B = A + TX * g.nz;
    const int f = blockIdx.z, ky = blockIdx.y, kx0 = blockIdx.x * TX;
    const int ncol = min(TX, g.nxh - kx0);
    const long long base = (long long)f * g.NK + (long long)ky * g.nxh + kx0;
    const long long zs = (long long)g.ny * g.nxh;
    const double kyv = g.ky[ky];
    static_assert(sizeof(T) == 8, "the FP32-bulk form assembles its stages in k_stage_assemble_df");
    auto src = [&](int kz, int col) -> T2 {
        if (col >= ncol) return T2{0, 0};
        const long long gi = base + kz * zs + col;
        // every load first (independent, all in flight together), then the sums
        const double2 yv = __ldg(y + gi);
        const double lam = lam_at(g, ph, f, gi, g.kx[kx0 + col], kyv, g.kz[kz]);
        const double qv = (st.has_gamma && st.qin) ? __ldg(st.qin + gi) : 1.0;
        const unsigned mz = st.mI & ~st.mY;
        double2 zv[kMaxStages], fv[kMaxStages];
#pragma unroll
        for (int j = 0; j < kMaxStages; ++j) {
            zv[j] = fv[j] = make_double2(0.0, 0.0);
            if (j < st.n) {
                if ((mz >> j) & 1u) zv[j] = __ldg(st.z[j] + gi);
                if ((st.mE >> j) & 1u) fv[j] = __ldg(reinterpret_cast<const double2*>(st.f[j]) + gi);
            }
        }
        double2 r = yv;
        double2 zi = make_double2(0.0, 0.0);  // sum_j (dt A^I_ij) z_j, times lambda below
#pragma unroll
        for (int j = 0; j < kMaxStages; ++j) {
            if (j < st.n) {
                if ((st.mI >> j) & 1u) axpy(zi, cI_of(st, j), ((st.mY >> j) & 1u) ? yv : zv[j]);
                if ((st.mE >> j) & 1u) axpy(r, cE_of(st, j), fv[j]);
            }
        }
        axpy(r, lam, zi);
        if (st.qout) st.qout[gi] = 1.0 / (1.0 - qgamma_of(st) * lam);
        if (st.has_gamma) {
            const double q = st.qin ? qv : 1.0 / (1.0 - gamma_of(st) * lam);
            r.x *= q;
            r.y *= q;
        }
        if (zout) zout[gi] = r;
        return r;
    };
    auto dst = [&](int kz, int col, T2 v) {
        if (col < ncol) W[base + kz * zs + col] = v;
    };
    // few terms: few registers per element, so several elements' loads go out together
    cols_fft<+1, TX, false, (MAXT == 0 ? 4 : (MAXT <= 2 ? 2 : 1)), R16, PID>(g.pz, A, B, src, dst);
}

template <typename T>
void launch_z_stage(const Geo& g, const Phys& ph, const double2* y, const StageTerms& st, double2* zout, void* W,
                    cudaStream_t s) {
    using T2 = typename Cx<T>::t;
    const int TX = tuned_cols<T>(g, g.tx_z, g.nz, 2, 128 * 1024);
    const size_t sm = 2 * (size_t)TX * g.nz * sizeof(T2);
    dim3 grid((g.nxh + TX - 1) / TX, g.ny, 4);
    constexpr int MT = kMaxStages;
    PF_COL_SWITCH(T, g.pz, TX, set_smem(k_z_stage<T, TXC, R16C, PIDC, MT>, sm);
                  k_z_stage<T, TXC, R16C, PIDC, MT><<<grid, kThreads, sm, s>>>(g, ph, y, st, zout,
                                                                             reinterpret_cast<T2*>(W)));
}

// ---------------------------------------------------------------------------
// z pass: step completion, embedded local error, inverse FFT of the error
//   y_n = y + sum_i (dt b^I_i) lambda z_i + (dt b^E_i) f^E_i
//   LTE = sum_i (dt (b-bt)^I_i) lambda z_i + (dt (b-bt)^E_i) f^E_i
// ---------------------------------------------------------------------------
template <typename T, int TX, bool R16, int PID>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? 3 : 2) k_z_final(Geo g, Phys ph, const double2* __restrict__ y, StageTerms bt,
                                                      StageTerms dt, int want_lte, double2* __restrict__ ynew,
                                                      typename Cx<T>::t* __restrict__ W) {
    PF_SKIP_INACTIVE(g);
    if (y_swapped(g)) {
        double2* other = const_cast<double2*>(y);
        y = ynew;
        ynew = other;
    }
    using T2 = typename Cx<T>::t;
    extern __shared__ __align__(16) unsigned char smraw[];
    T2* A = reinterpret_cast<T2*>(smraw);
    T2* B = A + TX * g.nz;
    const int f = blockIdx.z, ky = blockIdx.y, kx0 = blockIdx.x * TX;
    const int ncol = min(TX, g.nxh - kx0);
    const long long base = (long long)f * g.NK + (long long)ky * g.nxh + kx0;
    const long long zs = (long long)g.ny * g.nxh;
    const double kyv = g.ky[ky];
    static_assert(sizeof(T) == 8, "the FP32-bulk form completes its steps in k_step_complete_df");
    auto combine = [&](int kz, int col) -> T2 {
        if (col >= ncol) return T2{0, 0};
        const long long gi = base + kz * zs + col;
        const unsigned lmI = want_lte ? dt.mI : 0u, lmE = want_lte ? dt.mE : 0u;
        const unsigned mI = bt.mI | lmI, mE = bt.mE | lmE, mz = mI & ~bt.mY;
        // every load first, then the sums
        const double2 yv = __ldg(y + gi);
        const double lam = lam_at(g, ph, f, gi, g.kx[kx0 + col], kyv, g.kz[kz]);
        double2 zv[kMaxStages], fv[kMaxStages];
#pragma unroll
        for (int j = 0; j < kMaxStages; ++j) {
            zv[j] = fv[j] = make_double2(0.0, 0.0);
            if (j < bt.n) {
                if ((mz >> j) & 1u) zv[j] = __ldg(bt.z[j] + gi);
                if ((mE >> j) & 1u) fv[j] = __ldg(reinterpret_cast<const double2*>(bt.f[j]) + gi);
            }
        }
        double2 r = yv;
        double2 l = make_double2(0.0, 0.0);
        double2 zr = make_double2(0.0, 0.0), zl = make_double2(0.0, 0.0);  // times lambda below
#pragma unroll
        for (int j = 0; j < kMaxStages; ++j) {
            if (j < bt.n) {
                const double2 zj = ((bt.mY >> j) & 1u) ? yv : zv[j];
                if ((bt.mI >> j) & 1u) axpy(zr, cI_of(bt, j), zj);
                if ((lmI >> j) & 1u) axpy(zl, cI_of(dt, j), zj);
                if ((bt.mE >> j) & 1u) axpy(r, cE_of(bt, j), fv[j]);
                if ((lmE >> j) & 1u) axpy(l, cE_of(dt, j), fv[j]);
            }
        }
        axpy(r, lam, zr);
        axpy(l, lam, zl);
        ynew[gi] = r;
        return l;
    };
    if (!want_lte) {
        for (int e = threadIdx.x; e < TX * g.nz; e += blockDim.x) combine(e / TX, e & (TX - 1));
        return;
    }
    auto dst = [&](int kz, int col, T2 v) {
        if (col < ncol) W[base + kz * zs + col] = v;
    };
    cols_fft<+1, TX, false, 1, R16, PID>(g.pz, A, B, combine, dst);
}

template <typename T>
void launch_z_final(const Geo& g, const Phys& ph, const double2* y, const StageTerms& bterm, const StageTerms& dterm,
                    int want_lte, double2* ynew, void* W, cudaStream_t s) {
    using T2 = typename Cx<T>::t;
    const int TX = tuned_cols<T>(g, g.tx_z, g.nz, 2, 128 * 1024);
    const size_t sm = 2 * (size_t)TX * g.nz * sizeof(T2);
    dim3 grid((g.nxh + TX - 1) / TX, g.ny, 4);
    PF_COL_SWITCH(T, g.pz, TX, set_smem(k_z_final<T, TXC, R16C, PIDC>, sm);
                  k_z_final<T, TXC, R16C, PIDC><<<grid, kThreads, sm, s>>>(g, ph, y, bterm, dterm, want_lte, ynew,
                                                                        reinterpret_cast<T2*>(W)));
}

}  // namespace pf
