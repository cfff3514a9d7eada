// Operand tables of the tensor-core P^2 step (step2d_tc.cuh): basis values
// (evaluation, mesh independent) and projection weights (scaled by 1/dx,
// 1/dy and the inverse mass), laid out per lane as the B fragments of
// mma.m16n8k8 (k = t and t + 4, n = g for lane = 4 g + t), each value split
// into a TF32 high part (low 13 bits cleared) and the FP32 remainder.
#pragma once
#include <cstdint>
#include <cstring>

#include "tables.cuh"

namespace crk {

// point of column n of evaluation tile nt (P^2, 3 Gauss points per direction)
//   tile 0: volume points q = n (q = a*3 + b)
//   tile 1: n = 2p: east point p, n = 2p+1: west point p, n = 6: volume q = 8
//   tile 2: n = 2p: north point p, n = 2p+1: south point p
//   other columns: no point (evaluated as the cell average, weight 0)
enum TcKind { TC_VOL = 0, TC_E = 1, TC_W = 2, TC_N = 3, TC_S = 4, TC_NONE = 5 };
inline void tc_point(int nt, int n, int* kind, int* idx) {
    *idx = 0;
    if (nt == 0) { *kind = TC_VOL; *idx = n; return; }
    if (n == 6 && nt == 1) { *kind = TC_VOL; *idx = 8; return; }
    if (n >= 6) { *kind = TC_NONE; return; }
    const int p = n / 2;
    *idx = p;
    if (nt == 1) *kind = (n & 1) ? TC_W : TC_E;
    else *kind = (n & 1) ? TC_S : TC_N;
}
// k column -> mode / point column permutation: k = t <-> 2t, k = t + 4 <-> 2t + 1
inline int tc_perm(int k) { return k < 4 ? 2 * k : 2 * (k - 4) + 1; }

inline float tf32_hi(float x) {
    uint32_t u;
    std::memcpy(&u, &x, 4);
    u &= 0xffffe000u;
    float r;
    std::memcpy(&r, &u, 4);
    return r;
}

// groups of the projection (k tile of evaluation tile nt, flux component,
// output tile): 0 (nt0,x)->V 1 (nt0,y)->V 2 (nt1,x)->F 3 (nt1,x)->V
// 4 (nt1,y)->V 5 (nt2,y)->F
constexpr int TC_NGROUP = 6;
constexpr int TC_TABLE_FLOATS = (3 + TC_NGROUP) * 32 * 4;

// table[tile][lane][4] = (b0 hi, b1 hi, b0 lo, b1 lo); tiles 0..2 evaluation,
// 3..8 projection groups
inline void tc_build_tables(double dx, double dy, float* table) {
    constexpr Tab2D<2, 0> tb = make_tab2d<2, 0>();
    const double rx = 1.0 / dx, ry = 1.0 / dy;
    auto put = [&](int tile, int lane, double v0, double v1) {
        float* o = table + (tile * 32 + lane) * 4;
        const float f0 = (float)v0, f1 = (float)v1;
        o[0] = tf32_hi(f0);
        o[1] = tf32_hi(f1);
        o[2] = f0 - o[0];
        o[3] = f1 - o[1];
    };
    // evaluation: B[k][n] = phi_{perm(k)}(point(nt, n)); mode >= 6 is padding
    for (int nt = 0; nt < 3; ++nt)
        for (int lane = 0; lane < 32; ++lane) {
            const int g = lane >> 2, t = lane & 3;
            double v[2];
            for (int h = 0; h < 2; ++h) {
                const int m = tc_perm(t + 4 * h);
                int kind, idx;
                tc_point(nt, g, &kind, &idx);
                double val = 0.0;
                if (m < 6) {
                    switch (kind) {
                        case TC_VOL: val = tb.phi[idx][m]; break;
                        case TC_E: val = tb.tE[idx][m]; break;
                        case TC_W: val = tb.tW[idx][m]; break;
                        case TC_N: val = tb.tN[idx][m]; break;
                        case TC_S: val = tb.tS[idx][m]; break;
                        default: val = m == 0 ? 1.0 : 0.0; break;   // no point: the cell average
                    }
                }
                v[h] = val;
            }
            put(nt, lane, v[0], v[1]);
        }
    // projection: B[k][n] = weight of point(nt, perm(k)), component, mode n
    const int gnt[TC_NGROUP] = {0, 0, 1, 1, 1, 2};
    const int gcomp[TC_NGROUP] = {0, 1, 0, 0, 1, 1};
    const int gout[TC_NGROUP] = {1, 1, 0, 1, 1, 0};   // 0: face part F, 1: volume part V
    for (int gi = 0; gi < TC_NGROUP; ++gi)
        for (int lane = 0; lane < 32; ++lane) {
            const int g = lane >> 2, t = lane & 3;
            const int m = g;   // output column = mode
            double v[2];
            for (int h = 0; h < 2; ++h) {
                int kind, idx;
                tc_point(gnt[gi], tc_perm(t + 4 * h), &kind, &idx);
                double w = 0.0;
                if (m < 6) {
                    const double cm = tb.cm[m];
                    const bool vol = kind == TC_VOL, xc = gcomp[gi] == 0;
                    if (gout[gi] == 1 && vol) w = -cm * (xc ? rx * tb.gx[idx][m] : ry * tb.gy[idx][m]);
                    if (gout[gi] == 0 && !vol) {
                        if (kind == TC_E && xc) w = cm * rx * tb.pE[idx][m];
                        if (kind == TC_W && xc) w = -cm * rx * tb.pW[idx][m];
                        if (kind == TC_N && !xc) w = cm * ry * tb.pN[idx][m];
                        if (kind == TC_S && !xc) w = -cm * ry * tb.pS[idx][m];
                    }
                }
                v[h] = w;
            }
            put(3 + gi, lane, v[0], v[1]);
        }
}

}  // namespace crk
