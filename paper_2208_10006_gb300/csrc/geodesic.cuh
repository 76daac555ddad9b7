// Geodesic launch direction of ray `id` (Sec. II-A.1, Fig. 1), decoded on the
// fly so that no direction table is stored or read from memory.
//
// Class-I frequency-N subdivision of the icosahedron, flat then projected:
// ids [0, 12) are the vertices; [12, 12 + 30(N-1)) the interior points of the
// sorted edges (N-1 per edge, k = 1..N-1); the rest the interior points of
// the sorted faces, (N-1)(N-2)/2 per face, rows i = 1..N-2 (outer), columns
// j = 1..N-1-i. Computed in FP64.
#pragma once
#include "sbr_internal.cuh"

namespace sbr {

__device__ __forceinline__ d3 geodesic_dir(const Ico& ico, int N, uint32_t id) {
    d3 p;
    if (id < 12u) {
        p = ld3(ico.v[id]);
    } else {
        uint32_t r = id - 12u;
        uint32_t ne = 30u * (uint32_t)(N - 1);
        if (r < ne) {
            uint32_t e = r / (uint32_t)(N - 1);
            uint32_t k = r % (uint32_t)(N - 1) + 1u;
            d3 a = ld3(ico.v[ico.e[e][0]]), b = ld3(ico.v[ico.e[e][1]]);
            p = a + (b - a) * ((double)k / N);
        } else {
            r -= ne;
            uint32_t m = (uint32_t)((int64_t)(N - 1) * (N - 2) / 2);
            uint32_t f = r / m;
            uint32_t l = r % m;
            // row i holds N-1-i points; rows before i hold (i-1)(N-1) - i(i-1)/2
            // solve for the largest i with that count <= l, then fix rounding
            double b2 = 2.0 * N - 1.0;
            double disc = b2 * b2 - 8.0 * (double)l - 8.0 * (N - 1);
            int64_t i = (int64_t)floor((b2 - sqrt(fmax(disc, 0.0))) / 2.0);
            if (i < 1) i = 1;
            auto before = [N](int64_t ii) { return (ii - 1) * (int64_t)(N - 1) - ii * (ii - 1) / 2; };
            while (i > 1 && before(i) > (int64_t)l) --i;
            while (i < N - 2 && before(i + 1) <= (int64_t)l) ++i;
            int64_t j = (int64_t)l - before(i) + 1;
            d3 a = ld3(ico.v[ico.f[f][0]]), b = ld3(ico.v[ico.f[f][1]]), c = ld3(ico.v[ico.f[f][2]]);
            p = a + ((b - a) * ((double)i / N) + (c - a) * ((double)j / N));
        }
    }
    return unit(p);
}

}  // namespace sbr
