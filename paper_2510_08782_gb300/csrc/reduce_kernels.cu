// Reductions and small vector kernels of the solver (Sec. 2.3; Alg. 1-3).
//
// Inner products are FP64-accurate and deterministic: every thread accumulates a compensated
// partial sum (FP32 data: a double-float pair, products split exactly with an FMA; FP64 data:
// Neumaier summation), CTAs combine their threads in FP64 in a fixed tree order and write one
// partial per CTA; a single-CTA pass sums the partials in a fixed order. The grid size is fixed,
// so results do not depend on scheduling.
//
// The NGMRES least squares (Alg. 1, "arg min") is solved from its Gram data in one CTA: the normal
// matrix G_ij = <g_q - g_i, g_q - g_j> = c - a_i - a_j + M_ij and right-hand side -(c - a_i)
// are diagonalised by cyclic Jacobi rotations in FP64 and eigenvalues below 1e-14 max are dropped.
#include <cuda_runtime.h>

#include <atomic>

#include "kernels.h"

namespace ga {

namespace {

struct AccF {  // double-float accumulator for FP32 products
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add_prod(float a, float b) {
    const float p = a * b;
    const float e = fmaf(a, b, -p);
    const float s = hi + p;
    const float bb = s - hi;
    const float err = (hi - (s - bb)) + (p - bb);
    hi = s;
    lo += err + e;
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

struct AccD {  // Neumaier accumulator for FP64 products
  double s = 0.0, c = 0.0;
  __device__ __forceinline__ void add_prod(double a, double b) {
    const double p = a * b;
    const double t = s + p;
    c += (fabs(s) >= fabs(p)) ? (s - t) + p : (p - t) + s;
    s = t;
  }
  __device__ __forceinline__ double value() const { return s + c; }
};

template <typename T> struct AccOf;
template <> struct AccOf<float> { using type = AccF; };
template <> struct AccOf<double> { using type = AccD; };

// Sum x over the CTA (fixed order); result valid in thread 0.
__device__ __forceinline__ double block_sum(double x) {
  __shared__ double red[kThreads / 32];
  for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = x;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x < 32) {
    r = threadIdx.x < kThreads / 32 ? red[threadIdx.x] : 0.0;
    for (int off = 16; off > 0; off >>= 1) r += __shfl_down_sync(0xffffffffu, r, off);
  }
  return r;
}

__device__ __forceinline__ double block_max(double x) {
  __shared__ double red[kThreads / 32];
  for (int off = 16; off > 0; off >>= 1) x = fmax(x, __shfl_down_sync(0xffffffffu, x, off));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = x;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x < 32) {
    r = threadIdx.x < kThreads / 32 ? red[threadIdx.x] : 0.0;
    for (int off = 16; off > 0; off >>= 1) r = fmax(r, __shfl_down_sync(0xffffffffu, r, off));
  }
  return r;
}

// Per-CTA partial sums of <a, b_k> for k < count (count <= NB).
// Each thread visits i, i + stride, i + 2 stride, ... in order; U consecutive visits load their
// operands before any of them is accumulated, so (1 + count) U loads are in flight per thread while
// every accumulator still receives its products in the same order.
template <typename T, int NB>
__device__ __forceinline__ void dots_body(const T* __restrict__ a, const T* const* b, int count, long long len,
                                          double* __restrict__ partial) {
  using Acc = typename AccOf<T>::type;
  constexpr int U = NB <= 4 ? 4 : (NB <= 8 ? 2 : 1);
  Acc acc[NB];
  const long long stride = (long long)gridDim.x * blockDim.x;
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  for (; i + (U - 1) * stride < len; i += U * stride) {
    T av[U], bv[U][NB];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      av[u] = a[i + u * stride];
#pragma unroll
      for (int k = 0; k < NB; ++k) bv[u][k] = k < count ? b[k][i + u * stride] : T(0);
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int k = 0; k < NB; ++k)
        if (k < count) acc[k].add_prod(av[u], bv[u][k]);
  }
  for (; i < len; i += stride) {
    const T av = a[i];
#pragma unroll
    for (int k = 0; k < NB; ++k)
      if (k < count) acc[k].add_prod(av, b[k][i]);
  }
#pragma unroll
  for (int k = 0; k < NB; ++k) {
    if (k < count) {
      const double s = block_sum(acc[k].value());
      if (threadIdx.x == 0) partial[(long long)k * gridDim.x + blockIdx.x] = s;
    }
  }
}

template <typename T, int NB>
__global__ void __launch_bounds__(kThreads)
k_dots(const T* __restrict__ a, PtrList<T> b, int count, long long len, double* __restrict__ partial) {
  dots_body<T, NB>(a, b.p, count, len, partial);
}

// ---- window ring of the device-driven solve ---------------------------------------------------
__device__ __forceinline__ int ring_slot(int head, int i, int W1) { return (((head - i) % W1) + W1) % W1; }
__device__ __forceinline__ int ring_head(const ResCtl* c, int W1) { return ring_slot(c->head, 0, W1); }
// entries of the ring that take part: all m, or the min(m, W1 - 1) a push keeps
__device__ __forceinline__ int ring_count(const ResCtl* c, int W1, int keep) {
  const int m = min(max(c->m, 0), W1);
  return keep ? min(m, W1 - 1) : m;
}

// Chunk `chunk` (16 products) of out = [<a, first>, <a, ring entry 0>, ...].
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_dots_ring(const T* __restrict__ a, const T* __restrict__ first, const T* __restrict__ ring, long long stride,
            const ResCtl* __restrict__ c, int W1, int keep, int chunk, long long len, double* __restrict__ partial) {
  const int count = 1 + ring_count(c, W1, keep), base = 16 * chunk;
  const int cnt = min(16, count - base);
  if (cnt <= 0) return;
  const int head = ring_head(c, W1);
  const T* b[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const int e = base + k;
    b[k] = (k >= cnt) ? nullptr : (e == 0 ? first : ring + (long long)ring_slot(head, e - 1, W1) * stride);
  }
  dots_body<T, 16>(a, b, cnt, len, partial + (long long)base * gridDim.x);
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
k_maxabs(const T* __restrict__ x, long long len, double* __restrict__ partial) {
  T m = T(0);  // max of |x| is exact in the element type (and independent of the visiting order)
  int bad = 0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  for (; i + 3 * stride < len; i += 4 * stride) {  // four loads in flight per thread
    T v4[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) v4[u] = fabs(x[i + u * stride]);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (!(v4[u] <= T(3.0e38))) bad = 1;  // NaN or Inf
      else m = v4[u] > m ? v4[u] : m;
    }
  }
  for (; i < len; i += stride) {
    const T v = fabs(x[i]);
    if (!(v <= T(3.0e38))) bad = 1;
    else m = v > m ? v : m;
  }
  const int anybad = __syncthreads_or(bad);
  const double r = block_max((double)m);
  if (threadIdx.x == 0) partial[blockIdx.x] = anybad ? __longlong_as_double(0x7ff8000000000000LL) : r;
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
k_mismatch(const T* __restrict__ mT, const T* __restrict__ m1, T* __restrict__ lam, long long len,
           double* __restrict__ partial) {
  using Acc = typename AccOf<T>::type;
  Acc acc;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < len;
       i += (long long)gridDim.x * blockDim.x) {
    const T r = m1[i] - mT[i];
    if (lam) lam[i] = r;
    acc.add_prod(r, r);
  }
  const double s = block_sum(acc.value());
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// out[k] = sum_b partial[k * nblocks + b], k < count: one warp per output, each lane sums a fixed
// strided subset in FP64 (Neumaier), then a fixed shuffle tree; deterministic.
__device__ __forceinline__ void sum_partials_body(const double* __restrict__ partial, int count, int nblocks,
                                                  double* __restrict__ out) {
  const int k = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (k >= count) return;
  double s = 0.0, c = 0.0;
  for (int b = lane; b < nblocks; b += 32) {
    const double p = partial[(long long)k * nblocks + b];
    const double t = s + p;
    c += (fabs(s) >= fabs(p)) ? (s - t) + p : (p - t) + s;
    s = t;
  }
  s += c;
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  if (lane == 0) out[k] = s;
}

__global__ void k_sum_partials(const double* __restrict__ partial, int count, int nblocks,
                               double* __restrict__ out) {
  sum_partials_body(partial, count, nblocks, out);
}

__global__ void k_sum_partials_ring(const double* __restrict__ partial, const ResCtl* __restrict__ c, int W1,
                                    int keep, int nblocks, double* __restrict__ out) {
  sum_partials_body(partial, 1 + ring_count(c, W1, keep), nblocks, out);
}

__global__ void k_max_partials(const double* __restrict__ partial, int nblocks, double* __restrict__ out) {
  double m = 0.0;
  int bad = 0;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
    const double p = partial[b];
    if (!(p <= 1.0e300)) bad = 1;
    else m = fmax(m, p);
  }
  const int anybad = __syncthreads_or(bad);
  const double r = block_max(m);
  if (threadIdx.x == 0) out[0] = anybad ? __longlong_as_double(0x7ff8000000000000LL) : r;
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
k_axpy(T* __restrict__ y, const T* __restrict__ x, const T* __restrict__ s, T a, long long len) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < len;
       i += (long long)gridDim.x * blockDim.x)
    y[i] = x[i] + a * s[i];
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
k_axpy_dev(T* __restrict__ y, const T* __restrict__ x, const T* __restrict__ s, const double* __restrict__ a,
           long long len) {
  const T av = (T)*a;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < len;
       i += (long long)gridDim.x * blockDim.x)
    y[i] = x[i] + av * s[i];
}

// out (+)= q + sum_{k < m} beta_k (q - v_k) for one chunk of at most 16 vectors
template <typename T>
__device__ __forceinline__ void combine_body(T* __restrict__ out, const T* __restrict__ q, const T* const* v,
                                             const double* __restrict__ beta, int m, int accumulate, long long len) {
  T bt[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) bt[k] = k < m ? (T)beta[k] : T(0);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < len;
       i += (long long)gridDim.x * blockDim.x) {
    const T qi = q[i];
    T acc = accumulate ? out[i] : qi;
#pragma unroll
    for (int k = 0; k < 16; ++k)
      if (k < m) acc += bt[k] * (qi - v[k][i]);
    out[i] = acc;
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
k_combine(T* __restrict__ out, const T* __restrict__ q, PtrList<T> v, const double* __restrict__ beta,
          int m, int accumulate, long long len) {
  combine_body<T>(out, q, v.p, beta, m, accumulate, len);
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
k_combine_ring(T* __restrict__ out, const T* __restrict__ q, const T* __restrict__ ring, long long stride,
               const ResCtl* __restrict__ c, int W1, const double* __restrict__ beta, int chunk, long long len) {
  const int m = ring_count(c, W1, 0), base = 16 * chunk;
  const int cnt = min(16, m - base);
  if (cnt <= 0 && chunk > 0) return;
  const int head = ring_head(c, W1);
  const T* v[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) v[k] = k < cnt ? ring + (long long)ring_slot(head, base + k, W1) * stride : nullptr;
  combine_body<T>(out, q, v, beta + base, cnt, chunk > 0 ? 1 : 0, len);
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
k_ring_store(T* __restrict__ ring, long long stride, const ResCtl* __restrict__ c, int W1, const T* __restrict__ src,
             long long len) {
  if (c->status != 0) return;
  T* dst = ring + (long long)ring_slot(ring_head(c, W1) + 1, 0, W1) * stride;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < len;
       i += (long long)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

// Cyclic Jacobi eigen-solve of the m x m normal equations (m <= kMaxWin) by one warp, with G, U and
// the right-hand side in shared memory. The rotations are applied one after another; the lanes share
// the row, column and eigenvector updates of each rotation. Every element receives the same
// operations in the same order as in a one-thread loop, and the scalar sums are taken by lane 0, so
// the result does not depend on the warp width.
__global__ void __launch_bounds__(32) k_lsq(int m, const double* __restrict__ dots, const double* __restrict__ M,
                                            int ldm, double* __restrict__ beta, double* __restrict__ info,
                                            const ResCtl* __restrict__ ctl) {
  if (ctl) {  // device-driven solve: m is the window size on the device
    if (ctl->status != 0) return;
    m = min(max(ctl->m, 1), min(ldm, kMaxWin));
  }
  extern __shared__ double sh[];
  double* G = sh;              // m * m
  double* U = sh + m * m;      // m * m
  double* r = sh + 2 * m * m;  // m
  __shared__ double s_scal[2];  // off-diagonal mass, Frobenius norm
  __shared__ int s_stop;
  const int lane = threadIdx.x;
  const double c = dots[0];
  for (int e = lane; e < m * m; e += 32) {
    const int i = e / m, j = e % m;
    G[e] = c - dots[1 + i] - dots[1 + j] + M[i * ldm + j];
    U[e] = (i == j) ? 1.0 : 0.0;
  }
  for (int i = lane; i < m; i += 32) r[i] = c - dots[1 + i];
  __syncwarp();
  for (int e = lane; e < m * m; e += 32) {  // symmetrise against rounding of the expansion
    const int i = e / m, j = e % m;
    if (j > i) {
      const double s = 0.5 * (G[i * m + j] + G[j * m + i]);
      G[i * m + j] = s;
      G[j * m + i] = s;
    }
  }
  __syncwarp();
  if (lane == 0) {
    double fro = 0.0;
    for (int i = 0; i < m * m; ++i) fro += G[i] * G[i];
    s_scal[1] = fro;
  }
  int sweep = 0;
  for (; sweep < 60; ++sweep) {
    __syncwarp();
    if (lane == 0) {
      double off = 0.0;
      for (int i = 0; i < m; ++i)
        for (int j = i + 1; j < m; ++j) off += 2.0 * G[i * m + j] * G[i * m + j];
      s_stop = (off <= 1e-30 * s_scal[1] || off == 0.0) ? 1 : 0;
    }
    __syncwarp();
    if (s_stop) break;
    for (int p = 0; p < m; ++p)
      for (int q = p + 1; q < m; ++q) {
        const double apq = G[p * m + q];
        if (apq == 0.0) continue;
        const double app = G[p * m + p], aqq = G[q * m + q];
        const double theta = (aqq - app) / (2.0 * apq);
        const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        const double cs = 1.0 / sqrt(t * t + 1.0), sn = t * cs;
        __syncwarp();
        for (int k = lane; k < m; k += 32) {  // G <- J^T G J, columns first
          const double gkp = G[k * m + p], gkq = G[k * m + q];
          G[k * m + p] = cs * gkp - sn * gkq;
          G[k * m + q] = sn * gkp + cs * gkq;
        }
        __syncwarp();
        for (int k = lane; k < m; k += 32) {
          const double gpk = G[p * m + k], gqk = G[q * m + k];
          G[p * m + k] = cs * gpk - sn * gqk;
          G[q * m + k] = sn * gpk + cs * gqk;
        }
        for (int k = lane; k < m; k += 32) {  // U <- U J
          const double ukp = U[k * m + p], ukq = U[k * m + q];
          U[k * m + p] = cs * ukp - sn * ukq;
          U[k * m + q] = sn * ukp + cs * ukq;
        }
        __syncwarp();
      }
  }
  __syncwarp();
  if (lane != 0) return;
  double lmax = 0.0;
  for (int i = 0; i < m; ++i) lmax = fmax(lmax, G[i * m + i]);
  const double thr = 1e-14 * lmax;
  for (int i = 0; i < m; ++i) beta[i] = 0.0;
  int rank = 0;
  for (int k = 0; k < m; ++k) {
    const double lam = G[k * m + k];
    if (!(lam > thr)) continue;
    ++rank;
    double proj = 0.0;
    for (int i = 0; i < m; ++i) proj += U[i * m + k] * r[i];
    const double coef = -proj / lam;
    for (int i = 0; i < m; ++i) beta[i] += coef * U[i * m + k];
  }
  if (info) {
    info[0] = (double)rank;
    info[1] = (double)sweep;
    info[2] = lmax;
  }
}

__global__ void k_gram_push(double* __restrict__ M, int ldm, int mkeep, const double* __restrict__ row,
                            const ResCtl* __restrict__ ctl) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (ctl) {  // device-driven solve: keep min(m, W1 - 1) entries
    if (ctl->status != 0) return;
    mkeep = min(max(ctl->m, 0), ldm - 1);
  }
  // shift the kept block down-right by one, in place from the bottom-right corner
  for (int i = mkeep - 1; i >= 0; --i)
    for (int j = mkeep - 1; j >= 0; --j) M[(i + 1) * ldm + (j + 1)] = M[i * ldm + j];
  M[0] = row[0];
  for (int i = 0; i < mkeep; ++i) {
    M[(i + 1) * ldm] = row[1 + i];
    M[i + 1] = row[1 + i];
  }
}

inline unsigned grid_for(long long n) {
  long long b = (n + kThreads - 1) / kThreads;
  const long long cap = 152LL * 8;
  return (unsigned)(b < 1 ? 1 : (b < cap ? b : cap));
}

}  // namespace

template <typename T>
cudaError_t launch_dots(const T* a, const T* const* b, int count, long long len, double* partial, double* out,
                        cudaStream_t st) {
  if (count < 1 || count > kMaxDots) return cudaErrorInvalidValue;
  for (int base = 0; base < count; base += 16) {
    PtrList<T> pl;
    const int cnt = (count - base) < 16 ? (count - base) : 16;
    for (int k = 0; k < 16; ++k) pl.p[k] = k < cnt ? b[base + k] : nullptr;
    note_launches(1);
    if (cnt <= 4)
      k_dots<T, 4><<<kRedBlocks, kThreads, 0, st>>>(a, pl, cnt, len, partial + (long long)base * kRedBlocks);
    else if (cnt <= 8)
      k_dots<T, 8><<<kRedBlocks, kThreads, 0, st>>>(a, pl, cnt, len, partial + (long long)base * kRedBlocks);
    else
      k_dots<T, 16><<<kRedBlocks, kThreads, 0, st>>>(a, pl, cnt, len, partial + (long long)base * kRedBlocks);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  note_launches(1);
  // one warp per product, at most 32 warps per block
  k_sum_partials<<<(count + 31) / 32, 32 * (count < 32 ? count : 32), 0, st>>>(partial, count, kRedBlocks, out);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_maxabs(const T* x, long long len, double* partial, double* out, cudaStream_t st) {
  note_launches(1);
  k_maxabs<T><<<kRedBlocks, kThreads, 0, st>>>(x, len, partial);
  note_launches(1);
  k_max_partials<<<1, kThreads, 0, st>>>(partial, kRedBlocks, out);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_mismatch(const T* mT, const T* m1, T* lam, long long len, double* partial, double* out,
                            cudaStream_t st) {
  note_launches(1);
  k_mismatch<T><<<kRedBlocks, kThreads, 0, st>>>(mT, m1, lam, len, partial);
  note_launches(1);
  k_sum_partials<<<1, 32, 0, st>>>(partial, 1, kRedBlocks, out);
  return cudaGetLastError();
}

cudaError_t launch_sum_partials(const double* partial, int count, int nblocks, double* out, cudaStream_t st) {
  note_launches(1);
  k_sum_partials<<<1, 32 * count, 0, st>>>(partial, count, nblocks, out);
  return cudaGetLastError();
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_fill(T* __restrict__ y, T value, long long len) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len; i += (long long)gridDim.x * blockDim.x)
    y[i] = value;
}

template <typename T>
cudaError_t launch_fill(T* y, double value, long long len, cudaStream_t st) {
  note_launches(1);
  k_fill<T><<<grid_for(len), kThreads, 0, st>>>(y, (T)value, len);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_axpy(T* y, const T* x, const T* s, double a, long long len, cudaStream_t st) {
  note_launches(1);
  k_axpy<T><<<grid_for(len), kThreads, 0, st>>>(y, x, s, (T)a, len);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_combine(T* out, const T* q, const T* const* v, const double* beta, int m, long long len,
                           cudaStream_t st) {
  if (m < 1) return cudaMemcpyAsync(out, q, sizeof(T) * len, cudaMemcpyDeviceToDevice, st);
  for (int base = 0; base < m; base += 16) {
    PtrList<T> pl;
    const int cnt = (m - base) < 16 ? (m - base) : 16;
    for (int k = 0; k < 16; ++k) pl.p[k] = k < cnt ? v[base + k] : nullptr;
    note_launches(1);
    k_combine<T><<<grid_for(len), kThreads, 0, st>>>(out, q, pl, beta + base, cnt, base > 0 ? 1 : 0, len);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

namespace {
cudaError_t lsq_smem_limit() {
  constexpr size_t kMaxSmem = sizeof(double) * (2 * kMaxWin * kMaxWin + kMaxWin);
  static std::atomic<bool> attr{false};
  if (!attr.load()) {  // one process-wide setting, the largest size any call needs
    cudaError_t e = cudaFuncSetAttribute(k_lsq, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxSmem);
    if (e != cudaSuccess) return e;
    attr.store(true);
  }
  return cudaSuccess;
}
}  // namespace

cudaError_t launch_lsq(int m, const double* dots, const double* M, int ldm, double* beta, double* info,
                       cudaStream_t st) {
  if (m < 1 || m > kMaxWin) return cudaErrorInvalidValue;
  cudaError_t e = lsq_smem_limit();
  if (e != cudaSuccess) return e;
  note_launches(1);
  k_lsq<<<1, 32, sizeof(double) * (2 * m * m + m), st>>>(m, dots, M, ldm, beta, info, nullptr);
  return cudaGetLastError();
}

cudaError_t launch_gram_push(double* M, int ldm, int mkeep, const double* row, cudaStream_t st) {
  note_launches(1);
  k_gram_push<<<1, 32, 0, st>>>(M, ldm, mkeep, row, nullptr);
  return cudaGetLastError();
}

// ---- ring variants of the device-driven solve ---------------------------------------------------
template <typename T>
cudaError_t launch_axpy_dev(T* y, const T* x, const T* s, const double* a, long long len, cudaStream_t st) {
  note_launches(1);
  k_axpy_dev<T><<<grid_for(len), kThreads, 0, st>>>(y, x, s, a, len);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_dots_ring(const T* a, const T* first, const T* ring, long long stride, const ResCtl* c, int W1,
                             int keep, long long len, double* partial, double* out, cudaStream_t st) {
  if (W1 < 1 || 1 + W1 > kMaxDots) return cudaErrorInvalidValue;
  for (int chunk = 0; 16 * chunk < 1 + W1; ++chunk) {
    note_launches(1);
    k_dots_ring<T><<<kRedBlocks, kThreads, 0, st>>>(a, first, ring, stride, c, W1, keep, chunk, len, partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  note_launches(1);
  const int most = 1 + W1;
  k_sum_partials_ring<<<(most + 31) / 32, 32 * (most < 32 ? most : 32), 0, st>>>(partial, c, W1, keep, kRedBlocks,
                                                                               out);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_combine_ring(T* out, const T* q, const T* ring, long long stride, const ResCtl* c, int W1,
                                const double* beta, long long len, cudaStream_t st) {
  if (W1 < 1 || W1 > kMaxWin) return cudaErrorInvalidValue;
  for (int chunk = 0; 16 * chunk < W1; ++chunk) {
    note_launches(1);
    k_combine_ring<T><<<grid_for(len), kThreads, 0, st>>>(out, q, ring, stride, c, W1, beta, chunk, len);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <typename T>
cudaError_t launch_ring_store(T* ring, long long stride, const ResCtl* c, int W1, const T* src, long long len,
                              cudaStream_t st) {
  note_launches(1);
  k_ring_store<T><<<grid_for(len), kThreads, 0, st>>>(ring, stride, c, W1, src, len);
  return cudaGetLastError();
}

cudaError_t launch_lsq_ring(const ResCtl* c, int W1, const double* dots, const double* M, double* beta, double* info,
                            cudaStream_t st) {
  if (W1 < 1 || W1 > kMaxWin) return cudaErrorInvalidValue;
  cudaError_t e = lsq_smem_limit();
  if (e != cudaSuccess) return e;
  note_launches(1);
  k_lsq<<<1, 32, sizeof(double) * (2 * W1 * W1 + W1), st>>>(W1, dots, M, W1, beta, info, c);
  return cudaGetLastError();
}

cudaError_t launch_gram_push_ring(double* M, int W1, const ResCtl* c, const double* row, cudaStream_t st) {
  note_launches(1);
  k_gram_push<<<1, 32, 0, st>>>(M, W1, 0, row, c);
  return cudaGetLastError();
}

#define GA_INST(T)                                                                                   \
  template cudaError_t launch_dots<T>(const T*, const T* const*, int, long long, double*, double*,    \
                                      cudaStream_t);                                                  \
  template cudaError_t launch_maxabs<T>(const T*, long long, double*, double*, cudaStream_t);         \
  template cudaError_t launch_mismatch<T>(const T*, const T*, T*, long long, double*, double*,        \
                                          cudaStream_t);                                              \
  template cudaError_t launch_axpy<T>(T*, const T*, const T*, double, long long, cudaStream_t);       \
  template cudaError_t launch_fill<T>(T*, double, long long, cudaStream_t);                          \
  template cudaError_t launch_combine<T>(T*, const T*, const T* const*, const double*, int, long long, \
                                         cudaStream_t);                                              \
  template cudaError_t launch_axpy_dev<T>(T*, const T*, const T*, const double*, long long, cudaStream_t); \
  template cudaError_t launch_dots_ring<T>(const T*, const T*, const T*, long long, const ResCtl*, int, int, \
                                           long long, double*, double*, cudaStream_t);                \
  template cudaError_t launch_combine_ring<T>(T*, const T*, const T*, long long, const ResCtl*, int,     \
                                              const double*, long long, cudaStream_t);                \
  template cudaError_t launch_ring_store<T>(T*, long long, const ResCtl*, int, const T*, long long,     \
                                            cudaStream_t);
GA_INST(float)
GA_INST(double)
#undef GA_INST

}  // namespace ga
