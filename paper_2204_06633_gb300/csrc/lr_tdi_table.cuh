// Michelson chain tables (Eqs. tdi1 and tdi2), built at compile time from the spacecraft
// sequences of the two chains of X; Y and Z follow from the cyclic map 1->2->3->1.
#pragma once
#include "lr_internal.h"

namespace lr {

// link order 12, 23, 31, 13, 32, 21 (receiver, emitter)
__host__ __device__ constexpr int link_of(int r, int s)
{
    return (r == 1 && s == 2) ? 0 : (r == 2 && s == 3) ? 1 : (r == 3 && s == 1) ? 2
         : (r == 1 && s == 3) ? 3 : (r == 3 && s == 2) ? 4 : (r == 2 && s == 1) ? 5 : -1;
}

__host__ __device__ constexpr int cyc(int i, int times)
{
    return times == 0 ? i : cyc(i % 3 + 1, times - 1);
}

// X = sum_{q=0..Q} D_{a_0..a_q} y_{a_q a_{q+1}}  -  sum_{q=0..Q} D_{b_0..b_q} y_{b_q b_{q+1}}
// with a = 1 3 1 2 1 2 1 3 1 and b = 1 2 1 3 1 3 1 2 1: q = 0..3 reproduces the eight terms of
// X1 and q = 4..7 the eight added by X2, in the printed order.
__host__ __device__ constexpr TdiTab make_tdi_tab()
{
    TdiTab t{};
    const int seq[2][9] = {{1, 3, 1, 2, 1, 2, 1, 3, 1}, {1, 2, 1, 3, 1, 3, 1, 2, 1}};
    for (int ch = 0; ch < 3; ++ch)
        for (int c = 0; c < 2; ++c)
            for (int q = 0; q < CHAIN_TERMS; ++q) {
                int a0 = cyc(seq[c][q], ch), a1 = cyc(seq[c][q + 1], ch);
                t.link[ch][c][q] = (signed char)link_of(a0, a1);
                if (q == 0) {
                    t.pair[ch][c][q] = -1;
                } else {
                    int p0 = cyc(seq[c][q - 1], ch), p1 = cyc(seq[c][q], ch);
                    t.pair[ch][c][q] = (signed char)link_of(p0, p1);
                }
            }
    return t;
}

}  // namespace lr
