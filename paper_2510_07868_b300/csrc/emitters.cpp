// Emitter table of next-event estimation (the paper's experiments run with it on,
// Sec. 5): every triangle whose material emits and whose area is positive, in the
// caller's triangle order, with the CDF of choosing one by area.
#include <cmath>
#include <cstring>

#include "emitters.h"

namespace nrrs {

namespace {

double tri_area(const float* t) {
    const double e1[3] = {(double)t[3] - t[0], (double)t[4] - t[1], (double)t[5] - t[2]};
    const double e2[3] = {(double)t[6] - t[0], (double)t[7] - t[1], (double)t[8] - t[2]};
    const double c[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2],
                         e1[0] * e2[1] - e1[1] * e2[0]};
    return 0.5 * std::sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
}

float as_float(uint32_t u) {
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}

}  // namespace

// The CDF entry of emitter k is the FP32 rounding of (sum of the first k + 1 areas) / A,
// summed in FP64 in triangle order, and the last entry is 1: a uniform u in [0, 1) picks
// the first k with u < cdf[k].  Edges are kept in FP32 as the triangle array keeps them.
EmitterHost build_emitters(const float* tri, int n_tri, const int32_t* tri_mat,
                           const nrrs_material* mats) {
    EmitterHost e;
    std::vector<double> area;
    for (int i = 0; i < n_tri; ++i) {
        const nrrs_material& m = mats[tri_mat[i]];
        if (!(m.Le[0] > 0.0f || m.Le[1] > 0.0f || m.Le[2] > 0.0f)) continue;
        const float* t = tri + 9 * (size_t)i;
        const double a = tri_area(t);
        if (!(a > 0.0)) continue;
        area.push_back(a);
        e.area += a;
        e.tri.push_back(make_float4(t[0], t[1], t[2], as_float((uint32_t)tri_mat[i])));
        e.tri.push_back(make_float4(t[3] - t[0], t[4] - t[1], t[5] - t[2], 0.0f));
        e.tri.push_back(make_float4(t[6] - t[0], t[7] - t[1], t[8] - t[2], 0.0f));
    }
    double run = 0.0;
    for (size_t k = 0; k < area.size(); ++k) {
        run += area[k];
        e.cdf.push_back(k + 1 == area.size() ? 1.0f : (float)(run / e.area));
    }
    return e;
}

}  // namespace nrrs
