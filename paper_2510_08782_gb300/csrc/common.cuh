// Shared types of the GB300 GA-NGMRES library (internal).
#pragma once

#include <cstddef>
#include <cstdint>

#if defined(__CUDACC__)
#include <cuda_runtime.h>
#define GA_HD __host__ __device__ __forceinline__
#else
#define GA_HD inline
struct float2 { float x, y; };
struct double2 { double x, y; };
#endif

namespace ga {

template <typename T> struct CxT;
template <> struct CxT<float> { using type = float2; };
template <> struct CxT<double> { using type = double2; };
template <typename T> using cx = typename CxT<T>::type;

template <typename T> GA_HD cx<T> mk(T x, T y) { cx<T> r; r.x = x; r.y = y; return r; }
template <typename C> GA_HD C cadd(C a, C b) { C r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename C> GA_HD C csub(C a, C b) { C r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
template <typename C> GA_HD C cmul(C a, C b) {
  C r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}
template <typename C> GA_HD C cconj(C a) { C r; r.x = a.x; r.y = -a.y; return r; }
// multiply by -i: (x + i y)(-i) = y - i x
template <typename C> GA_HD C cmul_negi(C a) { C r; r.x = a.y; r.y = -a.x; return r; }
template <typename C, typename T> GA_HD C cscale(C a, T s) { C r; r.x = a.x * s; r.y = a.y * s; return r; }

// Internal 3-axis grid. A 2D problem of size (N0, N1) is stored as (1, N0, N1); vector component
// c always points along internal axis 3 - dim + c. Axis 2 is contiguous.
struct Grid {
  int dim;
  int n[3];
  int n2h;                // n[2] / 2 + 1 (half spectrum along the contiguous axis)
  long long nvox;         // n0 * n1 * n2
  long long nhalf;        // n0 * n1 * n2h
  int sl_bz = 8;          // brick depth (z voxels per thread) of the FP32 3D state steps
  int sl_bz_adj = 8;      // the same for the adjoint steps
  GA_HD int axis_of(int c) const { return 3 - dim + c; }
};

// Mixed-radix factorisation of one FFT length (radices 2, 3, 4, 5, 8).
struct FftPlan {
  int n;
  int ns;
  int radix[24];
};

}  // namespace ga
