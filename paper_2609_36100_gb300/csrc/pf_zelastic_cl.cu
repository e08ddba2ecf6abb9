// Elastic pass (Green's contraction of Eq. u_gov, Sec. 4.2) as a cluster of
// three CTAs, one per h field, on a compiled z plan.
//
// Each CTA holds one field of TX kx columns in a [kz][col] tile of its own
// shared memory, so a column row is TX * 8 bytes of one field (128 bytes at
// TX = 16) and a 640-point column of one field needs 80 KB where the
// three-field tile of the single-CTA forms needs 240 KB.  The CTA runs the
// forward z transform of its field; after a cluster barrier the three CTAs
// share the contraction e^_v = sum_q (B_vq / N) h^_q: every wave number is
// owned by one thread of the cluster, which reads h^_0..2 from the three
// tiles (two of them in the peers' shared memory) and writes e^_0..2 back in
// place, so B(k) is read or formed once per wave number; after a second
// cluster barrier each CTA runs the inverse transform of its field.
//
// Launch order pairs ky with ny - ky (adjacent clusters), so the mirrored
// rows of the octant table of B(k)/N are read while still in L2.
#include <cooperative_groups.h>

#include "pf_yz.cuh"

namespace cg = cooperative_groups;

namespace pf {

// ky of the b-th cluster row: 0, ny-1, 1, ny-2, ... (a permutation of 0..ny-1)
__device__ __forceinline__ int ky_paired(int b, int ny) { return (b & 1) ? ny - ((b + 1) >> 1) : (b >> 1); }

template <int NT>
constexpr int elastic_cluster_min_blocks() {
    // registers for two CTAs of 640 threads (51 a thread), else 64 a thread
    return NT >= 512 ? 2 : (65536 / (NT * 64) > 8 ? 8 : 65536 / (NT * 64));
}

template <int TX, int PID, int NT>
__global__ void __cluster_dims__(3, 1, 1) __launch_bounds__(NT, elastic_cluster_min_blocks<NT>())
    k_z_elastic_cluster(Geo g, Phys ph, float2* __restrict__ H) {
    // the flag is the same for the three CTAs: a cluster returns as a whole
    PF_SKIP_INACTIVE(g);
    using T2 = float2;
    using Fwd = typename FixedPlan<PID>::Rad;
    using Inv = Reversed<Fwd>;
    constexpr int N = FixedPlan<PID>::N;
    constexpr int RF = RadInfo<Fwd>::first, RL = RadInfo<Fwd>::last;
    constexpr int E = N * TX;
    cg::cluster_group cl = cg::this_cluster();
    const int f = (int)cl.block_rank();  // the field of this CTA
    extern __shared__ __align__(16) unsigned char smraw[];
    T2* S = reinterpret_cast<T2*>(smraw);  // [N][TX] of field f
    const int ky = ky_paired(blockIdx.y, g.ny), kx0 = (blockIdx.x / 3) * TX;
    const int ncol = min(TX, g.nxh - kx0);
    const long long fb = (long long)f * g.NK + (long long)ky * g.nxh + kx0;
    const long long zs = (long long)g.ny * g.nxh;
    const T2* tw = twiddles<T2>(g.pz);
    {
        auto ld = [&](int, int kz, int col) -> T2 { return col < ncol ? H[fb + kz * zs + col] : T2{0.f, 0.f}; };
        auto st = [&](int, int kz, int col, T2 v) { S[kz * TX + col] = v; };
        tile_stage_io<RF, -1, TX, N, 1, 1, NT>(tw, ld, st);
    }
    __syncthreads();
    tile_stages_inplace<-1, TX, N, RF, 1, NT>(S, tw, typename DropFirst<Fwd>::type{});
    cl.sync();  // the three forward transforms are complete
    {
        T2* S0 = cl.map_shared_rank(S, 0);
        T2* S1 = cl.map_shared_rank(S, 1);
        T2* S2 = cl.map_shared_rank(S, 2);
        const float invN = g.invN32;
        const PhysT<float>& pt = phys_t<float>(ph);
        const float kyv = kval<float>(g, 1, ky);
        const float* bt = g.btab;
        const int hy = g.ny / 2 + 1;
        const long long tn = (long long)(g.nz / 2 + 1) * hy * g.nxh;
        const long long trow = (long long)(ky <= g.ny / 2 ? ky : g.ny - ky) * g.nxh + kx0;
        // two wave numbers per iteration, every load of both issued first
        // (the reads of the peers' tiles are the long-latency ones); one where
        // the registers are bounded for two CTAs of 512 or more threads
        constexpr int CU = NT >= 512 ? 1 : 2;
        for (int e0 = f * NT + (int)threadIdx.x; e0 < E; e0 += 3 * NT * CU) {
            T2 h[CU][3];
            float bv[CU][6];
            bool ok[CU];
#pragma unroll
            for (int u = 0; u < CU; ++u) {
                const int e = e0 + u * 3 * NT;
                const int kz = e / TX, col = e - kz * TX;
                ok[u] = e < E && col < ncol;
                if (ok[u]) {
                    h[u][0] = S0[e];
                    h[u][1] = S1[e];
                    h[u][2] = S2[e];
                    if (bt) {
                        const long long ti = (long long)(kz <= g.nz / 2 ? kz : g.nz - kz) * hy * g.nxh + trow + col;
#pragma unroll
                        for (int m = 0; m < 6; ++m) bv[u][m] = __ldg(bt + m * tn + ti);
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < CU; ++u) {
                if (!ok[u]) continue;
                const int e = e0 + u * 3 * NT;
                float Bm[3][3];
                float sc = invN;
                if (bt) {
                    Bm[0][0] = bv[u][0];
                    Bm[0][1] = Bm[1][0] = bv[u][1];
                    Bm[0][2] = Bm[2][0] = bv[u][2];
                    Bm[1][1] = bv[u][3];
                    Bm[1][2] = Bm[2][1] = bv[u][4];
                    Bm[2][2] = bv[u][5];
                    sc = 1.f;
                } else {
                    const int kz = e / TX, col = e - kz * TX;
                    elastic_kernel<float>(pt, kval<float>(g, 0, kx0 + col), kyv, kval<float>(g, 2, kz), Bm);
                }
                const T2 a = h[u][0], b = h[u][1], c = h[u][2];
                S0[e] = T2{(Bm[0][0] * a.x + Bm[0][1] * b.x + Bm[0][2] * c.x) * sc,
                           (Bm[0][0] * a.y + Bm[0][1] * b.y + Bm[0][2] * c.y) * sc};
                S1[e] = T2{(Bm[1][0] * a.x + Bm[1][1] * b.x + Bm[1][2] * c.x) * sc,
                           (Bm[1][0] * a.y + Bm[1][1] * b.y + Bm[1][2] * c.y) * sc};
                S2[e] = T2{(Bm[2][0] * a.x + Bm[2][1] * b.x + Bm[2][2] * c.x) * sc,
                           (Bm[2][0] * a.y + Bm[2][1] * b.y + Bm[2][2] * c.y) * sc};
            }
        }
    }
    cl.sync();  // every wave number contracted: no CTA reads a peer's tile after this
    // inverse: the reversed radix order (its first stage has NS = 1), in place
    // up to the last stage, which writes global memory
    tile_stage_inplace<RL, +1, TX, N, 1, 1, NT>(S, tw);
    tile_stages_inplace<+1, TX, N, RL, 1, NT>(S, tw, typename PlanInner<Inv>::type{});
    {
        auto ld = [&](int, int kz, int col) -> T2 { return S[kz * TX + col]; };
        auto st = [&](int, int kz, int col, T2 v) {
            if (col < ncol) H[fb + kz * zs + col] = v;
        };
        tile_stage_io<RF, +1, TX, N, N / RF, 1, NT>(tw, ld, st);
    }
}

template <int PID, int TX>
constexpr int elastic_cluster_threads() {
    constexpr int n = TX * FixedPlan<PID>::N / RadMax<typename FixedPlan<PID>::Rad>::value;
    return n > 1024 ? 1024 : (n + 31) / 32 * 32;
}

template <int PID>
static bool launch_cluster_plan(const Geo& g, const Phys& ph, void* H, int tuned, cudaStream_t s) {
    if constexpr (!fused_elastic_ok<PID>()) {
        return false;
    } else {
        constexpr int N = FixedPlan<PID>::N;
        // 16 columns (128-byte rows) unless the tuned width is 8
        const int TX = tuned == 8 ? 8 : 16;
        const size_t sm = (size_t)TX * N * sizeof(float2);
        if (sm > 200 * 1024) return false;
        dim3 grid(3 * ((g.nxh + TX - 1) / TX), g.ny, 1);
#define PF_ELC(TXC)                                                                                  \
    {                                                                                                \
        constexpr int NTC = elastic_cluster_threads<PID, TXC>();                                     \
        set_smem(k_z_elastic_cluster<TXC, PID, NTC>, sm);                                            \
        k_z_elastic_cluster<TXC, PID, NTC><<<grid, NTC, sm, s>>>(g, ph, reinterpret_cast<float2*>(H)); \
    }
        if (TX == 8)
            PF_ELC(8)
        else
            PF_ELC(16)
#undef PF_ELC
        return true;
    }
}

template <>
bool launch_z_elastic_cluster<float>(const Geo& g, const Phys& ph, void* H, int pid, cudaStream_t s) {
    switch (pid) {
        case 1: return launch_cluster_plan<1>(g, ph, H, g.tx_el, s);
        case 2: return launch_cluster_plan<2>(g, ph, H, g.tx_el, s);
        case 3: return launch_cluster_plan<3>(g, ph, H, g.tx_el, s);
        case 4: return launch_cluster_plan<4>(g, ph, H, g.tx_el, s);
        case 5: return launch_cluster_plan<5>(g, ph, H, g.tx_el, s);
        case 6: return launch_cluster_plan<6>(g, ph, H, g.tx_el, s);
        case 7: return launch_cluster_plan<7>(g, ph, H, g.tx_el, s);
        case 8: return launch_cluster_plan<8>(g, ph, H, g.tx_el, s);
        case 9: return launch_cluster_plan<9>(g, ph, H, g.tx_el, s);
        case 10: return launch_cluster_plan<10>(g, ph, H, g.tx_el, s);
        case 11: return launch_cluster_plan<11>(g, ph, H, g.tx_el, s);
        default: return false;
    }
}

// FP64 contexts keep the single-CTA forms
template <>
bool launch_z_elastic_cluster<double>(const Geo&, const Phys&, void*, int, cudaStream_t) {
    return false;
}

}  // namespace pf
