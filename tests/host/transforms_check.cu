// Host driver for tests/test_transforms_cpu.py: evaluates the library's
// moment transforms (lbm_core.cuh, host builds of the __host__ __device__
// functions) on vectors read from stdin and prints the results, so that the
// test can hold them to the plain matrix products of the d'Humieres basis.
// Input: 19 values f, then 19 values c (c[0] = c[3] = c[5] = 0).
// Output lines: m (one-lane), m (two-lane, lane x then lane y), f + M^T c
// (one-lane), f + M^T c (two-lane, lane x then lane y).
#include <cstdio>

#include "../../paper_1604_03478_gb300/csrc/lbm_core.cuh"

using namespace lbm;

static void print19(const float *v) {
    for (int i = 0; i < 19; ++i) std::printf("%.9e%c", v[i], i == 18 ? '\n' : ' ');
}

int main() {
    float f[19], c[19];
    for (int i = 0; i < 19; ++i)
        if (std::scanf("%f", &f[i]) != 1) return 1;
    for (int i = 0; i < 19; ++i)
        if (std::scanf("%f", &c[i]) != 1) return 1;
    float S[9], D[9], m[19];
    float2 f2[19], c2[19], S2[9], D2[9], m2[19];
    for (int i = 0; i < 19; ++i) {
        f2[i] = make_float2(f[i], -2.0f * f[i]);  // lane y: another vector
        c2[i] = make_float2(c[i], -2.0f * c[i]);
    }
    for (int P = 0; P < 9; ++P) {
        S[P] = f[pf(P)] + f[opp(pf(P))];
        D[P] = f[pf(P)] - f[opp(pf(P))];
        S2[P] = add2(f2[pf(P)], f2[opp(pf(P))]);
        D2[P] = sub2(f2[pf(P)], f2[opp(pf(P))]);
    }
    moments_shared(f[0], S, D, m);
    moments_shared2(f2[0], S2, D2, m2);
    print19(m);
    float mx[19], my[19];
    for (int i = 0; i < 19; ++i) { mx[i] = m2[i].x; my[i] = m2[i].y; }
    print19(mx);
    print19(my);
    float fo[19];
    for (int i = 0; i < 19; ++i) fo[i] = f[i];
    add_back_shared(fo, c);
    print19(fo);
    add_back_shared2(f2, c2);
    for (int i = 0; i < 19; ++i) { mx[i] = f2[i].x; my[i] = f2[i].y; }
    print19(mx);
    print19(my);
    return 0;
}
