// cx_labels.cu -- morphology labels of a colony: b sampled on a circle about
// the inoculum by bilinear interpolation of the cell-centred values (the
// branch count of the envelope is the number of circular runs of samples
// above the envelope level; the paper reads branch numbers off its figures,
// Sec. 3).
#include <math.h>

#include "cx_internal.h"

namespace cx {
namespace {

template <typename T>
__global__ void polar_kernel(const T *__restrict__ b, int nx, int ny, long long pitch, double dx,
                             double radius, int ns, double *__restrict__ out)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= ns) return;
    const double ang = 2.0 * 3.14159265358979323846 * (double)k / (double)ns;
    double x = radius * cos(ang) / dx + 0.5 * nx - 0.5;
    double y = radius * sin(ang) / dx + 0.5 * ny - 0.5;
    x = fmin(fmax(x, 0.0), (double)(nx - 1));
    y = fmin(fmax(y, 0.0), (double)(ny - 1));
    const int i0 = min((int)floor(x), nx - 1), j0 = min((int)floor(y), ny - 1);
    const int i1 = min(i0 + 1, nx - 1), j1 = min(j0 + 1, ny - 1);
    const double wx = x - i0, wy = y - j0;
    // the array is in pair order (cx_internal.h)
    const long long c0 = pair_col(i0), c1 = pair_col(i1);
    const double b00 = (double)b[(long long)j0 * pitch + c0], b01 = (double)b[(long long)j0 * pitch + c1];
    const double b10 = (double)b[(long long)j1 * pitch + c0], b11 = (double)b[(long long)j1 * pitch + c1];
    out[k] = (1.0 - wy) * ((1.0 - wx) * b00 + wx * b01) + wy * ((1.0 - wx) * b10 + wx * b11);
}

}  // namespace

cudaError_t launch_polar(int prec, const void *b, int nx, int ny, long long pitch, double dx,
                         double radius, int ns, double *out, cudaStream_t st)
{
    const int tb = 256, g = (ns + tb - 1) / tb;
    if (prec == CX_PREC_F64)
        polar_kernel<double><<<g, tb, 0, st>>>((const double *)b, nx, ny, pitch, dx, radius, ns, out);
    else
        polar_kernel<float><<<g, tb, 0, st>>>((const float *)b, nx, ny, pitch, dx, radius, ns, out);
    return cudaGetLastError();
}

}  // namespace cx
