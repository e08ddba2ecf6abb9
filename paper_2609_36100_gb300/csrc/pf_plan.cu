// Axis plans (radix schedules and division magic) and the x-pass CTA count.
#include "pf_xpass.cuh"

namespace pf {
int compiled_plan_len(int pid) { return fixed_plan_len(pid); }
int compiled_plan_count() { return kFixedPlans; }

// plan from an explicit radix order (each radix in {2,3,4,5,8,16}, product n)
bool make_axis_plan_radices(int n, const int* rad, int nr, AxisPlan& p) {
    if (nr < 1 || nr > kMaxRadices) return false;
    long long prod = 1;
    for (int s = 0; s < nr; ++s) {
        if (rad[s] != 2 && rad[s] != 3 && rad[s] != 4 && rad[s] != 5 && rad[s] != 8 && rad[s] != 16) return false;
        prod *= rad[s];
    }
    if (prod != n) return false;
    p.n = n;
    p.nst = nr;
    p.has16 = 0;
    for (int s = 0; s < nr; ++s)
        if (rad[s] == 16) p.has16 = 1;
    unsigned Ns = 1;
    for (int s = 0; s < nr; ++s) {
        p.rad[s] = rad[s];
        p.mulm[s] = magic_u32((unsigned)(n / rad[s]));
        p.mulN[s] = magic_u32(Ns);
        Ns *= (unsigned)rad[s];
    }
    return true;
}

// default schedule: the fewest stages, largest radices first -- radix-16
// stages (prefer16) or radix-8 ones, then a 8 / 4 (or 4*4 instead of 8*2,
// 8*4 instead of 16*2) or 2, then the 3s and 5s
bool make_axis_plan(int n, AxisPlan& p, bool prefer16) {
    int m = n, a = 0, b = 0, c = 0;
    while (m % 2 == 0) { m /= 2; ++a; }
    while (m % 3 == 0) { m /= 3; ++b; }
    while (m % 5 == 0) { m /= 5; ++c; }
    if (m != 1) return false;
    int r[kMaxRadices + 8];
    int nr = 0;
    if (prefer16) {
        int n16 = a / 4;
        int rem = a % 4;
        if (rem == 1 && n16 > 0) {
            --n16;
            rem = 5;
        }
        for (int i = 0; i < n16; ++i) r[nr++] = 16;
        if (rem == 5) {
            r[nr++] = 8;
            r[nr++] = 4;
        } else if (rem == 3) {
            r[nr++] = 8;
        } else if (rem == 2) {
            r[nr++] = 4;
        } else if (rem == 1) {
            r[nr++] = 2;
        }
    } else {
        int n8 = a / 3;
        const int rem = a % 3;
        bool two4 = false;
        if (rem == 1 && n8 > 0) {
            --n8;
            two4 = true;
        }
        for (int i = 0; i < n8; ++i) r[nr++] = 8;
        if (two4) {
            r[nr++] = 4;
            r[nr++] = 4;
        } else if (rem == 2) {
            r[nr++] = 4;
        } else if (rem == 1) {
            r[nr++] = 2;
        }
    }
    for (int i = 0; i < b; ++i) r[nr++] = 3;
    for (int i = 0; i < c; ++i) r[nr++] = 5;
    if (nr > kMaxRadices) return false;
    return make_axis_plan_radices(n, r, nr, p);
}

int x_pass_blocks(const Geo& g, int f64) {
    const int P = f64 ? x_rows<double>(g) : x_rows<float>(g);
    const int npairs = g.nz * g.ny / 2;
    return (npairs + P - 1) / P;
}

}  // namespace pf
