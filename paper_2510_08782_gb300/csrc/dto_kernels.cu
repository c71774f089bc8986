// Discretise-then-optimise gradient of the semi-Lagrangian advection objective (exact derivative of
// the discrete objective; the paper's own gradient optimises then discretises, Sec. 2.1).
//
// With m_{j+1} = A m_j, (A f)(x) = I[f](X-(x)), the backward sweep needs
//   the transpose of A (a scatter through the interpolation weights),
//   G_c(x) += coef r(x) (d_c I[m_j])(X-(x)), the derivative of the cubic interpolant with respect to
//     the departure point's coordinate along the axis of component c (grid units),
// and the chain rule through X-_a = x_a - (h_t/(2 h_a)) (v_a(x) + I[v_a](X*(x))), X*_b = x_b - h_t v_b / h_b:
//   out_a(y) = -(h_t/(2 h_a)) [G_a(y) + sum_x G_a(x) w(X*(x) -> y)]
//              + (h_t^2/(2 h_a)) sum_b (G_b(y)/h_b) (d_a I[v_b])(X*(y)).
// Scatters use atomic additions, so FP32 results depend on the order of the additions at the
// rounding level.
#include <cuda_runtime.h>

#include "kernels.h"

namespace ga {

namespace {

template <typename T> struct DTaps {
  int i[4];
  T w[4];
  T dw[4];  // d w / d t
};

template <typename T> __device__ __forceinline__ T dfloor(T x);
template <> __device__ __forceinline__ float dfloor<float>(float x) { return floorf(x); }
template <> __device__ __forceinline__ double dfloor<double>(double x) { return floor(x); }

// Cubic Lagrange weights on the nodes -1, 0, 1, 2 and their t-derivatives for grid index `base`
// displaced by `disp` cells on a periodic axis of n points.
template <typename T> __device__ __forceinline__ void make_dtaps(int base, T disp, int n, DTaps<T>& tp) {
  T fl = dfloor<T>(disp);
  const T t = disp - fl;
  fl = fmin(fmax(fl, T(-1048576)), T(1048576));
  int i0 = (base + (int)fl - 1) % n;
  if (i0 < 0) i0 += n;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    tp.i[k] = i0;
    i0 = (i0 + 1 == n) ? 0 : i0 + 1;
  }
  const T tp1 = t + T(1), tm1 = t - T(1), tm2 = t - T(2);
  const T sixth = T(1) / T(6);
  tp.w[0] = -t * tm1 * tm2 * sixth;
  tp.w[1] = tp1 * tm1 * tm2 * T(0.5);
  tp.w[2] = -tp1 * t * tm2 * T(0.5);
  tp.w[3] = tp1 * t * tm1 * sixth;
  const T t2 = t * t;
  tp.dw[0] = -(T(3) * t2 - T(6) * t + T(2)) * sixth;
  tp.dw[1] = (T(3) * t2 - T(4) * t - T(1)) * T(0.5);
  tp.dw[2] = -(T(3) * t2 - T(2) * t - T(2)) * T(0.5);
  tp.dw[3] = (T(3) * t2 - T(1)) * sixth;
}

// a single-tap stencil for the unused axis of a 2D grid
template <typename T> __device__ __forceinline__ void unit_taps(DTaps<T>& tp) {
  for (int k = 0; k < 4; ++k) {
    tp.i[k] = 0;
    tp.w[k] = T(0);
    tp.dw[k] = T(0);
  }
  tp.w[0] = T(1);
}

struct P3 {
  int i[3];
};
__device__ __forceinline__ P3 unflat(long long idx, int n1, int n2) {
  P3 p;
  p.i[2] = (int)(idx % n2);
  const long long q = idx / n2;
  p.i[1] = (int)(q % n1);
  p.i[0] = (int)(q / n1);
  return p;
}

template <typename T> __device__ __forceinline__ T twopi() { return T(6.283185307179586476925286766559); }

// Stencil of the point x + d (d: displacement in cells along the internal axes; 2D grids use axes 1, 2).
template <typename T, int DIM>
__device__ __forceinline__ void stencil(const Grid& g, const P3& p, const T* d, DTaps<T>* tp) {
  if (DIM == 3)
    make_dtaps<T>(p.i[0], d[0], g.n[0], tp[0]);
  else
    unit_taps<T>(tp[0]);
  make_dtaps<T>(p.i[1], d[1], g.n[1], tp[1]);
  make_dtaps<T>(p.i[2], d[2], g.n[2], tp[2]);
}
template <int DIM> __device__ __forceinline__ int na0() { return DIM == 3 ? 4 : 1; }

// G_c(x) += coef r(x) (d_c I[m])(x + disp(x)) for the dim components.
template <typename T, int DIM>
__global__ void __launch_bounds__(kThreads)
k_dto_accum(Grid g, const T* __restrict__ r, const T* __restrict__ m, const T* __restrict__ disp, T* __restrict__ G,
            T coef) {
  const long long nv = g.nvox;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < nv;
       idx += (long long)gridDim.x * blockDim.x) {
    const T rv = r[idx];
    if (rv == T(0)) continue;
    const P3 p = unflat(idx, g.n[1], g.n[2]);
    T d[3] = {T(0), T(0), T(0)};
    for (int c = 0; c < DIM; ++c) d[3 - DIM + c] = disp[c * nv + idx];
    DTaps<T> tp[3];
    stencil<T, DIM>(g, p, d, tp);
    T s[3] = {T(0), T(0), T(0)};  // derivatives along internal axes 0, 1, 2
    for (int a = 0; a < na0<DIM>(); ++a) {
      for (int b = 0; b < 4; ++b) {
        const T* row = m + ((size_t)tp[0].i[a] * g.n[1] + tp[1].i[b]) * g.n[2];
        T f = T(0), fx = T(0);
        for (int c = 0; c < 4; ++c) {
          const T val = row[tp[2].i[c]];
          f += tp[2].w[c] * val;
          fx += tp[2].dw[c] * val;
        }
        s[0] += tp[0].dw[a] * tp[1].w[b] * f;
        s[1] += tp[0].w[a] * tp[1].dw[b] * f;
        s[2] += tp[0].w[a] * tp[1].w[b] * fx;
      }
    }
    for (int c = 0; c < DIM; ++c) G[c * nv + idx] += coef * rv * s[3 - DIM + c];
  }
}

// out[taps of x + disp(x)] += w r(x): the transpose of the interpolation (out zeroed by the caller).
template <typename T, int DIM>
__global__ void __launch_bounds__(kThreads)
k_interp_scatter(Grid g, const T* __restrict__ r, const T* __restrict__ disp, T* __restrict__ out) {
  const long long nv = g.nvox;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < nv;
       idx += (long long)gridDim.x * blockDim.x) {
    const T rv = r[idx];
    if (rv == T(0)) continue;
    const P3 p = unflat(idx, g.n[1], g.n[2]);
    T d[3] = {T(0), T(0), T(0)};
    for (int c = 0; c < DIM; ++c) d[3 - DIM + c] = disp[c * nv + idx];
    DTaps<T> tp[3];
    stencil<T, DIM>(g, p, d, tp);
    for (int a = 0; a < na0<DIM>(); ++a)
      for (int b = 0; b < 4; ++b) {
        T* row = out + ((size_t)tp[0].i[a] * g.n[1] + tp[1].i[b]) * g.n[2];
        const T wab = tp[0].w[a] * tp[1].w[b] * rv;
        for (int c = 0; c < 4; ++c) atomicAdd(row + tp[2].i[c], wab * tp[2].w[c]);
      }
  }
}

// Local terms of the chain rule through the RK2 departure points (written, not accumulated):
// out_a(y) = -(h_t/(2 h_a)) G_a(y) + (h_t^2/(2 h_a)) sum_b (G_b(y)/h_b) (d_a I[v_b])(X*(y)).
template <typename T, int DIM>
__global__ void __launch_bounds__(kThreads)
k_dto_vel_local(Grid g, const T* __restrict__ v, const T* __restrict__ G, T* __restrict__ out, T ht) {
  const long long nv = g.nvox;
  T h[3];
  for (int a = 0; a < 3; ++a) h[a] = twopi<T>() / T(g.n[a]);
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < nv;
       idx += (long long)gridDim.x * blockDim.x) {
    const P3 p = unflat(idx, g.n[1], g.n[2]);
    T d[3] = {T(0), T(0), T(0)};
    for (int c = 0; c < DIM; ++c) {
      const int ax = 3 - DIM + c;
      d[ax] = -ht * v[c * nv + idx] / h[ax];
    }
    DTaps<T> tp[3];
    stencil<T, DIM>(g, p, d, tp);
    T acc[3] = {T(0), T(0), T(0)};  // sum_b (G_b / h_b) d_ax I[v_b] for each internal axis ax
    for (int b = 0; b < DIM; ++b) {
      const T gb = G[b * nv + idx] / h[3 - DIM + b];
      if (gb == T(0)) continue;
      const T* vb = v + b * nv;
      for (int a = 0; a < na0<DIM>(); ++a)
        for (int bb = 0; bb < 4; ++bb) {
          const T* row = vb + ((size_t)tp[0].i[a] * g.n[1] + tp[1].i[bb]) * g.n[2];
          T f = T(0), fx = T(0);
          for (int c = 0; c < 4; ++c) {
            const T val = row[tp[2].i[c]];
            f += tp[2].w[c] * val;
            fx += tp[2].dw[c] * val;
          }
          acc[0] += gb * tp[0].dw[a] * tp[1].w[bb] * f;
          acc[1] += gb * tp[0].w[a] * tp[1].dw[bb] * f;
          acc[2] += gb * tp[0].w[a] * tp[1].w[bb] * fx;
        }
    }
    for (int c = 0; c < DIM; ++c) {
      const int ax = 3 - DIM + c;
      out[c * nv + idx] = -(ht / (T(2) * h[ax])) * G[c * nv + idx] + (ht * ht / (T(2) * h[ax])) * acc[ax];
    }
  }
}

// The scatter term: out_a[taps of X*(x)] += -(h_t/(2 h_a)) G_a(x) w.
template <typename T, int DIM>
__global__ void __launch_bounds__(kThreads)
k_dto_vel_scatter(Grid g, const T* __restrict__ v, const T* __restrict__ G, T* __restrict__ out, T ht) {
  const long long nv = g.nvox;
  T h[3];
  for (int a = 0; a < 3; ++a) h[a] = twopi<T>() / T(g.n[a]);
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < nv;
       idx += (long long)gridDim.x * blockDim.x) {
    const P3 p = unflat(idx, g.n[1], g.n[2]);
    T d[3] = {T(0), T(0), T(0)};
    for (int c = 0; c < DIM; ++c) {
      const int ax = 3 - DIM + c;
      d[ax] = -ht * v[c * nv + idx] / h[ax];
    }
    DTaps<T> tp[3];
    stencil<T, DIM>(g, p, d, tp);
    for (int c = 0; c < DIM; ++c) {
      const T val = -(ht / (T(2) * h[3 - DIM + c])) * G[c * nv + idx];
      if (val == T(0)) continue;
      T* oc = out + c * nv;
      for (int a = 0; a < na0<DIM>(); ++a)
        for (int b = 0; b < 4; ++b) {
          T* row = oc + ((size_t)tp[0].i[a] * g.n[1] + tp[1].i[b]) * g.n[2];
          const T wab = tp[0].w[a] * tp[1].w[b] * val;
          for (int cc = 0; cc < 4; ++cc) atomicAdd(row + tp[2].i[cc], wab * tp[2].w[cc]);
        }
    }
  }
}

inline unsigned dto_grid(long long n) {
  long long b = (n + kThreads - 1) / kThreads;
  const long long cap = 152LL * 16;
  return (unsigned)(b < 1 ? 1 : (b < cap ? b : cap));
}

}  // namespace

template <typename T>
cudaError_t launch_dto_accum(const Grid& g, const T* r, const T* m, const T* disp, T* G, T coef, cudaStream_t st) {
  note_launches(1);
  if (g.dim == 3)
    k_dto_accum<T, 3><<<dto_grid(g.nvox), kThreads, 0, st>>>(g, r, m, disp, G, coef);
  else
    k_dto_accum<T, 2><<<dto_grid(g.nvox), kThreads, 0, st>>>(g, r, m, disp, G, coef);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_interp_scatter(const Grid& g, const T* r, const T* disp, T* out, cudaStream_t st) {
  note_launches(1);
  if (g.dim == 3)
    k_interp_scatter<T, 3><<<dto_grid(g.nvox), kThreads, 0, st>>>(g, r, disp, out);
  else
    k_interp_scatter<T, 2><<<dto_grid(g.nvox), kThreads, 0, st>>>(g, r, disp, out);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_dto_velocity(const Grid& g, const T* v, const T* G, T* out, T ht, cudaStream_t st) {
  note_launches(2);
  if (g.dim == 3) {
    k_dto_vel_local<T, 3><<<dto_grid(g.nvox), kThreads, 0, st>>>(g, v, G, out, ht);
    k_dto_vel_scatter<T, 3><<<dto_grid(g.nvox), kThreads, 0, st>>>(g, v, G, out, ht);
  } else {
    k_dto_vel_local<T, 2><<<dto_grid(g.nvox), kThreads, 0, st>>>(g, v, G, out, ht);
    k_dto_vel_scatter<T, 2><<<dto_grid(g.nvox), kThreads, 0, st>>>(g, v, G, out, ht);
  }
  return cudaGetLastError();
}

#define GA_DTO_INST(T)                                                                                   \
  template cudaError_t launch_dto_accum<T>(const Grid&, const T*, const T*, const T*, T*, T, cudaStream_t); \
  template cudaError_t launch_interp_scatter<T>(const Grid&, const T*, const T*, T*, cudaStream_t);      \
  template cudaError_t launch_dto_velocity<T>(const Grid&, const T*, const T*, T*, T, cudaStream_t);
GA_DTO_INST(float)
GA_DTO_INST(double)
#undef GA_DTO_INST

}  // namespace ga
