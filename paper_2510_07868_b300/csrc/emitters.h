// Host-side emitter table of next-event estimation (emitters.cpp).
#pragma once
#include <cstdint>
#include <vector>
#include <cuda_runtime.h>

#include "../../include/nrrs.h"

namespace nrrs {

struct EmitterHost {
    std::vector<float4> tri;  // 3 per emitter: (v0, material bits), (e1, 0), (e2, 0)
    std::vector<float> cdf;   // choice by area, last entry 1
    double area = 0.0;        // total emitter area
};

EmitterHost build_emitters(const float* tri, int n_tri, const int32_t* tri_mat,
                           const nrrs_material* mats);

}  // namespace nrrs
