// cx_batch_types.cuh -- device-side records of a batch (cx_batch.cu,
// cx_batch_kernels.cuh): the per-instance table entry and the state of the
// resident kernel's grid barrier.
#pragma once

#include "cx_stencil.cuh"

namespace cx {
namespace batch {

using stencil::CoefT;

template <typename T> struct InstDev {
    T *b[2];
    T *n[2];
    const T *s;
    int nx, ny;
    long long pitch;
    CoefT<T> k;
    float fth;     // FP32 envelope threshold (diagnostics)
    double bth;    // FP64 envelope threshold
    // per-step noise: sigma = sigma0 (1 + amp Delta(seed, cell, step)), Delta
    // of law `dist`, by the recipe of the state's precision
    uint64_t seed;
    T sigma0, amp;
    int dist;
};

// The per-step noise of instance I at time step `step`, as a single grid
// with the same seed draws it.
template <typename T>
__device__ __forceinline__ stencil::NoiseT<T> inst_noise(const InstDev<T> &I, uint64_t step)
{
    stencil::NoiseT<T> nz{};
    nz.seed = I.seed;
    nz.step = step;
    nz.dist = I.dist;
    nz.sigma0 = I.sigma0;
    nz.amp = I.amp;
    if constexpr (sizeof(T) == 4) nz.set_keys();
    return nz;
}

// State of the resident kernel's grid-wide barrier (cx_batch_kernels.cuh).
struct GridBarrier {
    unsigned count, gen;
    int err, pad;
};

}  // namespace batch
}  // namespace cx
