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
};

// State of the resident kernel's grid-wide barrier (cx_batch_kernels.cuh).
struct GridBarrier {
    unsigned count, gen;
    int err, pad;
};

}  // namespace batch
}  // namespace cx
