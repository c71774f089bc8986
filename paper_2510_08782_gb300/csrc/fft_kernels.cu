// Pencil FFT kernels: 1D spectral derivatives (fused with the body-force / divergence
// accumulation) and the passes of the real 3D FFT (Sec. 2.2: "two FFTs and a diagonal scaling").
//
// Every kernel stages a batch of pencils of one axis in shared memory (padded leading dimension
// to spread banks), runs the Stockham transform of fft_core.cuh, and writes back. Pencils along the
// contiguous axis are whole rows; pencils along the other axes are tiles of adjacent columns, so
// every global access is a contiguous row segment (coalesced). Two real pencils are packed into one
// complex pencil (z = a + i b):
//  * derivative: F^{-1}[i k~ F z] = d a + i d b exactly, because k~ is odd in k with the Nyquist
//    entry zeroed, so the derivative of a real pencil is real;
//  * real FFT rows: A_k = (Z_k + conj Z_{-k}) / 2, B_k = (Z_k - conj Z_{-k}) / (2 i).
// A 3D spectral derivative along one axis factorises into the 1D derivative along that axis (the
// transforms of the other axes cancel), so d/dx_c costs one pass, not a 3D FFT.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <unordered_set>
#include <type_traits>

#include "fft_core.cuh"
#include "kernels.h"

namespace ga {

namespace {

// Pencil element i of a work buffer lives at fpad<PS>(i) (one padding slot every 16 entries).
constexpr int PS = 4;
__device__ __forceinline__ int pd(int i) { return fpad<PS>(i); }

// (q, r) = (i / d, i % d) along a block-strided loop i = threadIdx.x, threadIdx.x + blockDim.x, ...:
// one division per thread, then constant steps (a runtime divisor costs a long instruction sequence
// per division).
struct StridedQR {
  int q, r, d, dq, dr;
  __device__ __forceinline__ StridedQR(int i, int d_) : d(d_) {
    q = i / d;
    r = i - q * d;
    dq = (int)blockDim.x / d;
    dr = (int)blockDim.x - dq * d;
  }
  __device__ __forceinline__ void next() {
    q += dq;
    r += dr;
    if (r >= d) {
      r -= d;
      ++q;
    }
  }
};

// Compile-time stage sequence for a fixed length N (radices from ct_next_radix, at most MAXR).
template <typename T, int N, int Ns, int MAXR> struct CtStages {
  __device__ __forceinline__ static cx<T>* run(cx<T>* a, cx<T>* b, int B, int ld, const cx<T>* tw) {
    if constexpr (Ns >= N) {
      return a;
    } else {
      constexpr int R = ct_next_radix(N / Ns, MAXR);
      constexpr int M = N / R;
      const int total = B * M;
      for (int t = threadIdx.x; t < total; t += blockDim.x) {
        const int p = t / M;
        const int j = t - p * M;
        stockham_butterfly_ct<T, N, R, Ns, PS>(a + p * ld, b + p * ld, j, tw);
      }
      __syncthreads();
      return CtStages<T, N, Ns * R, MAXR>::run(b, a, B, ld, tw);
    }
  }
};

template <typename T, int NC, int MAXR = 16>
__device__ cx<T>* run_fft(cx<T>* a, cx<T>* b, int N, int B, int ld, const FftPlan& plan,
                          const cx<T>* tw) {
  if constexpr (NC > 0) {
    return CtStages<T, NC, 1, MAXR>::run(a, b, B, ld, tw);
  }
  int Ns = 1;
  for (int s = 0; s < plan.ns; ++s) {
    const int R = plan.radix[s];
    const int M = N / R;
    const int total = B * M;
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
      const int p = t / M;
      const int j = t - p * M;
      stockham_butterfly<T, PS>(a + p * ld, b + p * ld, j, N, R, Ns, tw);
    }
    __syncthreads();
    cx<T>* tmp = a;
    a = b;
    b = tmp;
    Ns *= R;
  }
  return a;
}

// ---- forward transform with fused first and last stages (compile-time lengths) ------------------
template <typename T, int R> __device__ __forceinline__ void dft_r(cx<T>* v) {
  if constexpr (R == 2) dft2(v);
  else if constexpr (R == 3) dft3<T>(v);
  else if constexpr (R == 4) dft4(v);
  else if constexpr (R == 5) dft5<T>(v);
  else if constexpr (R == 16) dft16<T>(v);
  else dft8<T>(v);
}

// One Stockham stage (length N, radix R, span Ns) over B pencils, from `in` to `out`. The first stage
// (Ns == 1, all twiddles one) takes its inputs from load(p, i), element i of pencil p, so the staged
// real data need no separate packing pass; the last stage (Ns * R == N) stores fin(k, value) for
// frequency index k, so a diagonal scaling needs no separate pass either. With PFAST the first stage
// gives consecutive threads consecutive pencils (staged tiles whose pencils are adjacent columns).
template <typename T, int N, int R, int Ns, bool PFAST, typename Load, typename Fin>
__device__ __forceinline__ void fused_stage(Load& load, Fin& fin, const cx<T>* in, cx<T>* out, int B, int ld,
                                            const cx<T>* tw) {
  constexpr int M = N / R;
  constexpr bool pf = PFAST && Ns == 1;
  StridedQR qr(threadIdx.x, pf ? B : 1);  // pencil-fastest order: t = j * B + p
  for (int t = threadIdx.x; t < B * M; t += blockDim.x, qr.next()) {
    const int p = pf ? qr.r : t / M, j = pf ? qr.q : t - (t / M) * M;
    const int k = j % Ns;
    cx<T> v[R];
    if constexpr (Ns == 1) {
#pragma unroll
      for (int r = 0; r < R; ++r) v[r] = load(p, j + r * M);
    } else {
      const cx<T>* ip = in + p * ld;
      const int tstep = k * (N / (Ns * R));
      v[0] = ip[pd(j)];
#pragma unroll
      for (int r = 1; r < R; ++r) v[r] = cmul(ip[pd(j + r * M)], tw[r * tstep]);
    }
    dft_r<T, R>(v);
    const int base = (j - k) * R + k;
    cx<T>* op = out + p * ld;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int q = base + r * Ns;
      if constexpr (Ns * R == N)
        op[pd(q)] = fin(q, v[r]);
      else
        op[pd(q)] = v[r];
    }
  }
  __syncthreads();
}

// Forward transform of B pencils read through load(); stage s writes `out` and reads the previous
// stage's `out`. Returns the buffer holding fin(k, FFT(z)_k).
template <typename T, int N, int Ns, int MAXR, bool PFAST> struct FusedForward {
  template <typename Load, typename Fin>
  __device__ __forceinline__ static cx<T>* run(Load& load, Fin& fin, cx<T>* in, cx<T>* out, int B, int ld,
                                               const cx<T>* tw) {
    constexpr int R = ct_next_radix(N / Ns, MAXR);
    fused_stage<T, N, R, Ns, PFAST>(load, fin, in, out, B, ld, tw);
    if constexpr (Ns * R >= N)
      return out;
    else
      return FusedForward<T, N, Ns * R, MAXR, PFAST>::run(load, fin, out, in, B, ld, tw);
  }
};

// derivative wavenumber k~ of FFT index j of a length-L axis (zero at the Nyquist index)
template <typename T> __device__ __forceinline__ T ktilde(int j, int L) {
  if (2 * j == L) return T(0);
  return (2 * j < L) ? T(j) : T(j - L);
}

// conj(i k~ z) rotated for the conj-FFT-conj inverse: (-k~ z.y, -k~ z.x)
template <typename T> __device__ __forceinline__ void mult_ik_conj(cx<T>* r, int B, int L, int ld) {
  for (int idx = threadIdx.x; idx < B * L; idx += blockDim.x) {
    const int p = idx / L, j = idx - p * L;
    const T kt = ktilde<T>(j, L);
    const cx<T> z = r[p * ld + pd(j)];
    r[p * ld + pd(j)] = mk<T>(-kt * z.y, -kt * z.x);
  }
  __syncthreads();
}

template <typename T> __device__ __forceinline__ void load_tw(cx<T>* tw, const cx<T>* twg, int L) {
  for (int i = threadIdx.x; i < L; i += blockDim.x) tw[i] = twg[i];
}

// ---- asynchronous copies into shared memory ------------------------------------------------
__device__ __forceinline__ void cpa16(void* sdst, const void* gsrc) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"((unsigned)__cvta_generic_to_shared(sdst)),
               "l"(gsrc));
}
template <typename T> __device__ __forceinline__ void cpa_elem(T* sdst, const T* gsrc) {
  if constexpr (sizeof(T) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"((unsigned)__cvta_generic_to_shared(sdst)),
                 "l"(gsrc));
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"((unsigned)__cvta_generic_to_shared(sdst)),
                 "l"(gsrc));
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N> __device__ __forceinline__ void cpa_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// Copy `count` contiguous elements (16-byte chunks when vec) from global to shared memory.
template <typename T>
__device__ __forceinline__ void stage_contig(T* dst, const T* src, int count, bool vec) {
  constexpr int per = 16 / sizeof(T);
  if (vec) {
    for (int c = threadIdx.x; c < count / per; c += blockDim.x) cpa16(dst + c * per, src + c * per);
  } else {
    for (int e = threadIdx.x; e < count; e += blockDim.x) cpa_elem<T>(dst + e, src + e);
  }
}

// Copy W columns x [0, W) of L strided rows (row j at src + j * S) into dst[j * W + x]; columns at or
// beyond `valid` are not copied (the caller never reads them).
template <typename T>
__device__ __forceinline__ void stage_rows(T* dst, const T* src, int L, long long S, int W, int valid, bool vec) {
  constexpr int per = 16 / sizeof(T);
  if (vec) {  // W % per == 0, valid == W, 16-byte aligned rows
    const int cpr = W / per;
    StridedQR qr(threadIdx.x, cpr);
    for (int c = threadIdx.x; c < L * cpr; c += blockDim.x, qr.next())
      cpa16(dst + qr.q * W + qr.r * per, src + qr.q * S + qr.r * per);
  } else {
    StridedQR qr(threadIdx.x, W);
    for (int e = threadIdx.x; e < L * W; e += blockDim.x, qr.next())
      if (qr.r < valid) cpa_elem<T>(dst + e, src + qr.q * S + qr.r);
  }
}

// Shared-memory layout of the derivative kernels: twiddles, two complex work buffers of B pencils
// (the raw input block aliases the second), the raw multiplier block and the raw accumulator block.
template <typename T> struct DerivSmem {
  cx<T>* tw;
  cx<T>* a;
  cx<T>* b;
  T* raw;
  T* mult;
  T* acc;
  // regions are padded to an even number of complex entries so every region starts 16-byte aligned
  __device__ DerivSmem(unsigned char* base, int L, int B, int ld) {
    const size_t twn = ((size_t)L + 1) & ~(size_t)1, bufn = ((size_t)B * ld + 1) & ~(size_t)1;
    tw = reinterpret_cast<cx<T>*>(base);
    a = tw + twn;
    b = a + bufn;
    raw = reinterpret_cast<T*>(b);
    mult = reinterpret_cast<T*>(b + bufn);
    acc = mult + 2 * (size_t)B * L;
  }
};

// Operands of a derivative pass: out (+)= coef * mult * d f (one time step), or with PAIR
// out (+)= coef * mult * d f + coef2 * mult2 * d f2 (two time steps of the body force in one pass:
// f and f2 are the real and imaginary parts of one complex pencil, as two columns are otherwise).
// A null multiplier means 1. The sum is formed as two successive single passes would form it.
template <typename T> struct DerivIO {
  const T* f;
  const T* mult;
  const T* f2;
  const T* mult2;
  T* out;
  T coef, coef2;
  int accumulate;
};

template <typename T, bool PAIR>
__device__ __forceinline__ T deriv_out(const DerivIO<T>& io, const DerivSmem<T>& sm, int e, int plane, cx<T> z, T inv,
                                       bool odd) {
  if constexpr (PAIR) {
    T v1 = io.coef * (z.x * inv);
    if (io.mult) v1 *= sm.mult[e];
    if (io.accumulate) v1 += sm.acc[e];
    T v2 = io.coef2 * (-z.y * inv);
    if (io.mult2) v2 *= sm.mult[plane + e];
    return v2 + v1;
  } else {
    T val = io.coef * (odd ? -z.y * inv : z.x * inv);
    if (io.mult) val *= sm.mult[e];
    if (io.accumulate) val += sm.acc[e];
    return val;
  }
}

// ---- derivative along the contiguous axis (rows) --------------------------------------------
// Rows row0 .. row0 + 2B - 1 are one contiguous block: staged raw, then paired (2p, 2p+1) into
// complex pencils. PAIR: rows row0 .. row0 + B - 1 of f and of f2, paired (f row p, f2 row p).
template <typename T, int NC, bool PAIR>
__global__ void __launch_bounds__(kThreads)
k_deriv_rows(DerivIO<T> io, long long rows, int Lr, int B, int ld, FftPlan plan, const cx<T>* __restrict__ twg,
             int vec) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int L = NC > 0 ? NC : Lr;
  DerivSmem<T> sm(smem_raw, L, B, ld);
  constexpr int RPC = PAIR ? 1 : 2;  // rows of one field per complex pencil
  const long long row0 = (long long)blockIdx.x * RPC * B;
  const int nrows = (int)((rows - row0) < RPC * B ? (rows - row0) : RPC * B);
  const bool full = nrows == RPC * B && vec;
  const int plane = B * L;  // PAIR: offset of the second field's block in raw and mult
  stage_contig<T>(sm.raw, io.f + row0 * L, nrows * L, full);
  if (PAIR) stage_contig<T>(sm.raw + plane, io.f2 + row0 * L, nrows * L, full);
  cpa_commit();
  if (io.mult) stage_contig<T>(sm.mult, io.mult + row0 * L, nrows * L, full);
  if (PAIR && io.mult2) stage_contig<T>(sm.mult + plane, io.mult2 + row0 * L, nrows * L, full);
  if (io.accumulate) stage_contig<T>(sm.acc, io.out + row0 * L, nrows * L, full);
  cpa_commit();
  load_tw<T>(sm.tw, twg, L);
  cpa_wait<1>();
  __syncthreads();
  const T* raw = sm.raw;
  // element i of complex pencil p
  auto load = [&](int p, int i) {
    if constexpr (PAIR)
      return (p < nrows) ? mk<T>(raw[p * L + i], raw[plane + p * L + i]) : mk<T>(T(0), T(0));
    else
      return mk<T>((2 * p < nrows) ? raw[(2 * p) * L + i] : T(0), (2 * p + 1 < nrows) ? raw[(2 * p + 1) * L + i] : T(0));
  };
  cx<T>* r;
  if constexpr (NC > 0) {  // read straight from the staged block; i k~ applied on the way out
    auto fin = [&](int k, cx<T> z) {
      const T kt = ktilde<T>(k, L);
      return mk<T>(-kt * z.y, -kt * z.x);
    };
    r = FusedForward<T, NC, 1, 16, false>::run(load, fin, sm.b, sm.a, B, ld, sm.tw);  // sm.b holds the raw block
  } else {
    for (int idx = threadIdx.x; idx < B * L; idx += blockDim.x) {
      const int p = idx / L, j = idx - p * L;
      sm.a[p * ld + pd(j)] = load(p, j);
    }
    __syncthreads();
    r = run_fft<T, NC, 8>(sm.a, sm.b, L, B, ld, plan, sm.tw);
    mult_ik_conj<T>(r, B, L, ld);
  }
  cx<T>* o = (r == sm.a) ? sm.b : sm.a;
  cx<T>* r2 = run_fft<T, NC, 16>(r, o, L, B, ld, plan, sm.tw);
  cpa_wait<0>();
  __syncthreads();
  const T inv = T(1) / T(L);
  for (int idx = threadIdx.x; idx < nrows * L; idx += blockDim.x) {
    const int rr = idx / L, j = idx - rr * L;
    const cx<T> z = r2[(PAIR ? rr : (rr >> 1)) * ld + pd(j)];
    io.out[row0 * L + idx] = deriv_out<T, PAIR>(io, sm, idx, plane, z, inv, (rr & 1) != 0);
  }
}

// ---- derivative along a strided axis (tiles of adjacent columns) -------------------------------
// A tile holds W = 2B columns (PAIR: B columns of f and the same B columns of f2).
template <typename T, int NC, bool PAIR>
__global__ void __launch_bounds__(kThreads)
k_deriv_cols(DerivIO<T> io, int Lr, long long S, long long outer_stride, int nx, int B, int ld, FftPlan plan,
             const cx<T>* __restrict__ twg, int vec) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int L = NC > 0 ? NC : Lr;
  DerivSmem<T> sm(smem_raw, L, B, ld);
  const int W = PAIR ? B : 2 * B;
  const int x0 = blockIdx.x * W;
  const long long base = (long long)blockIdx.y * outer_stride + x0;
  const int valid = (nx - x0) < W ? (nx - x0) : W;
  const bool v16 = vec && valid == W;
  const int plane = W * L;
  stage_rows<T>(sm.raw, io.f + base, L, S, W, valid, v16);
  if (PAIR) stage_rows<T>(sm.raw + plane, io.f2 + base, L, S, W, valid, v16);
  cpa_commit();
  if (io.mult) stage_rows<T>(sm.mult, io.mult + base, L, S, W, valid, v16);
  if (PAIR && io.mult2) stage_rows<T>(sm.mult + plane, io.mult2 + base, L, S, W, valid, v16);
  if (io.accumulate) stage_rows<T>(sm.acc, io.out + base, L, S, W, valid, v16);
  cpa_commit();
  load_tw<T>(sm.tw, twg, L);
  cpa_wait<1>();
  __syncthreads();
  const T* raw = sm.raw;
  auto load = [&](int p, int i) {
    if constexpr (PAIR)
      return (p < valid) ? mk<T>(raw[i * W + p], raw[plane + i * W + p]) : mk<T>(T(0), T(0));
    else
      return mk<T>((2 * p < valid) ? raw[i * W + 2 * p] : T(0), (2 * p + 1 < valid) ? raw[i * W + 2 * p + 1] : T(0));
  };
  cx<T>* r;
  if constexpr (NC > 0) {  // read straight from the staged tile; i k~ applied on the way out
    auto fin = [&](int k, cx<T> z) {
      const T kt = ktilde<T>(k, L);
      return mk<T>(-kt * z.y, -kt * z.x);
    };
    r = FusedForward<T, NC, 1, 16, true>::run(load, fin, sm.b, sm.a, B, ld, sm.tw);  // sm.b holds the raw tile
  } else {
    StridedQR qr(threadIdx.x, B);
    for (int idx = threadIdx.x; idx < B * L; idx += blockDim.x, qr.next()) sm.a[qr.r * ld + pd(qr.q)] = load(qr.r, qr.q);
    __syncthreads();
    r = run_fft<T, NC, 8>(sm.a, sm.b, L, B, ld, plan, sm.tw);
    mult_ik_conj<T>(r, B, L, ld);
  }
  cx<T>* o = (r == sm.a) ? sm.b : sm.a;
  cx<T>* r2 = run_fft<T, NC, 16>(r, o, L, B, ld, plan, sm.tw);
  cpa_wait<0>();
  __syncthreads();
  const T inv = T(1) / T(L);
  StridedQR qr(threadIdx.x, W);
  for (int idx = threadIdx.x; idx < W * L; idx += blockDim.x, qr.next()) {
    const int j = qr.q, xx = qr.r;
    if (xx >= valid) continue;
    const cx<T> z = r2[(PAIR ? xx : (xx >> 1)) * ld + pd(j)];
    io.out[base + j * S + xx] = deriv_out<T, PAIR>(io, sm, idx, plane, z, inv, (xx & 1) != 0);
  }
}

// ---- register-resident derivative passes for 256-point axes -----------------------------------
// A 256-point transform as 16 x 16 (the four-step form): with n = q + 16 m and k = k2 + 16 k1,
//   X[k2 + 16 k1] = sum_q W16^(q k1) W256^(q k2) sum_m x[q + 16 m] W16^(m k2).
// 256 threads transform 16 complex pencils. In the load phase thread (p, q) holds x[q + 16 m] of
// pencil p (m = 0..15) in registers and applies the inner DFT16 over m and the twiddles W256^(q k2);
// one exchange through shared memory gives thread (p, k2) the values over q, whose DFT16 yields
// X[k2 + 16 k1] in registers. There the derivative symbol i k~ is applied, and the inverse runs the
// same steps backwards (DFT16 over k1 with conjugate weights, twiddles W256^(-n1 k2), one exchange,
// DFT16 over k2), leaving thread (p, n1) with the derivative at n1 + 16 n2, n2 = 0..15: the positions
// it loaded. Every index is a compile-time constant or a per-thread constant, and each element
// passes through shared memory twice. The exchange buffer holds entry (p, i, j) at p*273 + i*17 + j
// (complex units); the lanes of a warp differ either in p or in the fastest index of the global
// layout, and both strides are odd, so the exchanges are free of bank conflicts.
// ROWS: pencils along the contiguous axis (row p of the tile; the lanes of a half-warp cover
// consecutive elements); otherwise pencils along a strided axis (columns; the lanes of a half-warp
// cover consecutive columns). PAIR: pencil p is f + i f2 of one row/column (two time steps of the body
// force); otherwise pencil p packs rows/columns 2p and 2p + 1 of f.
constexpr int kX16P = 16 * 17 + 1;  // pencil stride of the exchange buffer
// Twiddles of the 256-point four-step transform as a 16 x 16 table, entry b * 16 + a = W256^(a b):
// thread x reads entry k * 16 + x for W256^(x k). The lanes of a half-warp share k and differ in x
// (pencils along rows) or read one entry (pencils along columns), so every read is free of bank
// conflicts (a table of W256^j indexed by x k would put lanes k entries apart).
template <typename T> __device__ __forceinline__ void load_tw256(cx<T>* tw, const cx<T>* __restrict__ twg) {
  for (int i = threadIdx.x; i < 256; i += blockDim.x) tw[i] = twg[(i >> 4) * (i & 15)];
}

template <typename T> __device__ __forceinline__ void idft16(cx<T>* a) {
#pragma unroll
  for (int i = 0; i < 16; ++i) a[i].y = -a[i].y;
  dft16<T>(a);
#pragma unroll
  for (int i = 0; i < 16; ++i) a[i].y = -a[i].y;
}

// The derivative of 16 complex pencils held in registers (see above): on entry thread (p, x) holds
// x[x + 16 m] of its pencil in a[m]; on return a[n2] holds 256 times the derivative at x + 16 n2.
// tw: the 16 x 16 twiddle table in shared memory (load_tw256); xp: this pencil's exchange area. Contains the CTA barriers of the two
// exchanges, so every thread of the CTA calls it.
template <typename T>
__device__ __forceinline__ void reg256_deriv(cx<T>* a, const cx<T>* tw, cx<T>* xp, int x) {
  // load phase: DFT16 over m, twiddles W256^(q k2), exchange
  dft16<T>(a);
#pragma unroll
  for (int k2 = 1; k2 < 16; ++k2) a[k2] = cmul(a[k2], tw[k2 * 16 + x]);
#pragma unroll
  for (int k2 = 0; k2 < 16; ++k2) xp[k2 * 17 + x] = a[k2];
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 16; ++q) a[q] = xp[x * 17 + q];  // thread now holds k2 = x over q
  dft16<T>(a);                                          // a[k1] = X[x + 16 k1]
  // derivative symbol i k~ (zero at the Nyquist index 128)
#pragma unroll
  for (int k1 = 0; k1 < 16; ++k1) {
    const int k = x + 16 * k1;
    const T kt = (k == 128) ? T(0) : (k < 128 ? T(k) : T(k - 256));
    a[k1] = mk<T>(-kt * a[k1].y, kt * a[k1].x);
  }
  // inverse: DFT16 over k1 with conjugate weights, twiddles W256^(-n1 k2), exchange, DFT16 over k2
  idft16<T>(a);  // a[n1]
#pragma unroll
  for (int n1 = 1; n1 < 16; ++n1) a[n1] = cmul(a[n1], cconj(tw[n1 * 16 + x]));
  __syncthreads();  // every thread has read its exchange entries
#pragma unroll
  for (int n1 = 0; n1 < 16; ++n1) xp[n1 * 17 + x] = a[n1];
  __syncthreads();
#pragma unroll
  for (int k2 = 0; k2 < 16; ++k2) a[k2] = xp[x * 17 + k2];  // thread holds n1 = x over k2
  idft16<T>(a);                                              // a[n2]: derivative at x + 16 n2
}

template <typename T, bool PAIR, bool ROWS>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 2)
k_deriv_reg256(DerivIO<T> io, long long npen, long long S, long long outer_stride, const cx<T>* __restrict__ twg) {
  constexpr int L = 256;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* tw = reinterpret_cast<cx<T>*>(smem_raw);  // W256^(a b) at b * 16 + a (load_tw256)
  cx<T>* xb = tw + L;                               // exchange buffer
  load_tw256<T>(tw, twg);
  const int t = threadIdx.x;
  const int p = ROWS ? (t >> 4) : (t & 15);  // complex pencil of the tile
  const int x = ROWS ? (t & 15) : (t >> 4);  // q, then k2, then n1
  constexpr int RP = PAIR ? 1 : 2;           // real rows/columns of f per complex pencil
  // global offset of element x of this thread's (first) real pencil; element x + 16 m is at
  // off + m * st16, the partner pencil (non-PAIR) pstride further
  const long long r0 = (long long)blockIdx.x * 16 * RP + RP * p;
  const bool v0 = r0 < npen, v1 = !PAIR && r0 + 1 < npen;
  const long long off = ROWS ? r0 * L + x : (long long)blockIdx.y * outer_stride + r0 + (long long)x * S;
  const long long st16 = ROWS ? 16 : 16 * S;
  const long long pstride = ROWS ? L : 1;
  // the operands of the output phase are read after the transforms: request their lines into L2 now
  if (v0) {
#pragma unroll 4
    for (int m = 0; m < 16; ++m) {
      const long long e = off + m * st16;
      if (io.mult) asm volatile("prefetch.global.L2 [%0];\n" ::"l"(io.mult + e));
      if (PAIR && io.mult2) asm volatile("prefetch.global.L2 [%0];\n" ::"l"(io.mult2 + e));
      if (io.accumulate) asm volatile("prefetch.global.L2 [%0];\n" ::"l"(io.out + e));
    }
  }
  cx<T> a[16];
  {
    const T* fp = io.f + off;
    const T* f2p = PAIR ? io.f2 + off : io.f + off + pstride;
#pragma unroll
    for (int m = 0; m < 16; ++m) {
      if (PAIR) {
        a[m] = v0 ? mk<T>(fp[0], f2p[0]) : mk<T>(T(0), T(0));
      } else {
        a[m] = mk<T>(v0 ? fp[0] : T(0), v1 ? f2p[0] : T(0));
      }
      fp += st16;
      f2p += st16;
    }
  }
  __syncthreads();  // twiddle table
  reg256_deriv<T>(a, tw, xb + p * kX16P, x);
  const T inv = T(1) / T(L);
  long long e = off;
#pragma unroll
  for (int n2 = 0; n2 < 16; ++n2, e += st16) {
    const T re = a[n2].x * inv, im = a[n2].y * inv;
    if (PAIR) {
      if (!v0) continue;
      T w1 = io.coef * re;
      if (io.mult) w1 *= io.mult[e];
      if (io.accumulate) w1 += io.out[e];
      T w2 = io.coef2 * im;
      if (io.mult2) w2 *= io.mult2[e];
      io.out[e] = w2 + w1;
    } else {
      if (v0) {
        T w = io.coef * re;
        if (io.mult) w *= io.mult[e];
        if (io.accumulate) w += io.out[e];
        io.out[e] = w;
      }
      if (v1) {
        T w = io.coef * im;
        if (io.mult) w *= io.mult[e + pstride];
        if (io.accumulate) w += io.out[e + pstride];
        io.out[e + pstride] = w;
      }
    }
  }
}

// FP32 form of the body force's two-step passes with their output operands staged: the two
// multipliers and the accumulator are copied into shared memory with cp.async as the CTA starts, so all
// of a tile's global reads are in flight while it transforms. The exchanges move the real and the
// imaginary parts in two rounds through a float buffer (half the shared memory of a complex one), which
// keeps three CTAs on an SM. Staging layouts: columns [n][c] (16 floats per row); rows [r][n] with a row
// pitch of 272 floats, so the two pencils a warp covers fall on different banks. (The one-field passes
// keep k_deriv_reg256: staging their single multiplier measured slower.)
__device__ __forceinline__ void xchg_split(float2* a, float* xr, int x) {
  // a[k] of this thread (fixed j = x) goes to entry (k, x); the thread then holds (x, q) for q = 0..15
#pragma unroll
  for (int k = 0; k < 16; ++k) xr[k * 17 + x] = a[k].x;
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 16; ++q) a[q].x = xr[x * 17 + q];
  __syncthreads();
#pragma unroll
  for (int k = 0; k < 16; ++k) xr[k * 17 + x] = a[k].y;
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 16; ++q) a[q].y = xr[x * 17 + q];
}

// reg256_deriv with the split exchanges (FP32).
__device__ __forceinline__ void reg256_deriv_split(float2* a, const float2* tw, float* xr, int x) {
  dft16<float>(a);
#pragma unroll
  for (int k2 = 1; k2 < 16; ++k2) a[k2] = cmul(a[k2], tw[k2 * 16 + x]);
  xchg_split(a, xr, x);  // thread holds k2 = x over q
  dft16<float>(a);       // a[k1] = X[x + 16 k1]
#pragma unroll
  for (int k1 = 0; k1 < 16; ++k1) {
    const int k = x + 16 * k1;
    const float kt = (k == 128) ? 0.f : (k < 128 ? float(k) : float(k - 256));
    a[k1] = make_float2(-kt * a[k1].y, kt * a[k1].x);
  }
  idft16<float>(a);  // a[n1]
#pragma unroll
  for (int n1 = 1; n1 < 16; ++n1) a[n1] = cmul(a[n1], cconj(tw[n1 * 16 + x]));
  __syncthreads();  // every thread has read the first exchange
  xchg_split(a, xr, x);  // thread holds n1 = x over k2
  idft16<float>(a);      // a[n2]: 256 times the derivative at x + 16 n2
}

template <bool ROWS> struct Reg256S {
  static constexpr int PITCH = ROWS ? 272 : 16;
  static constexpr int FIELD = ROWS ? 16 * PITCH : 256 * 16;  // floats of one staged field
  static constexpr size_t bytes() { return sizeof(float) * (2 * 256 + 16 * kX16P + 3 * FIELD); }
};

template <bool ROWS>
__global__ void __launch_bounds__(256, 3)
k_deriv_pair256s(DerivIO<float> io, long long npen, long long S, long long outer_stride,
                 const float2* __restrict__ twg, int vec) {
  using Z = Reg256S<ROWS>;
  constexpr int L = 256, PITCH = Z::PITCH, FIELD = Z::FIELD;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* tw = reinterpret_cast<float2*>(smem_raw);
  float* xr = reinterpret_cast<float*>(tw + L);
  float* stg = xr + 16 * kX16P;  // 16-byte aligned: 2 KB of twiddles + 16 * 273 floats
  const int t = threadIdx.x;
  const int p = ROWS ? (t >> 4) : (t & 15);
  const int x = ROWS ? (t & 15) : (t >> 4);
  // the tile: base offset and rows/columns present
  long long base;
  int valid;
  if (ROWS) {
    const long long r0 = (long long)blockIdx.x * 16;
    base = r0 * L;
    valid = (int)((npen - r0) < 16 ? (npen - r0) : 16);
  } else {
    const long long c0 = (long long)blockIdx.x * 16;
    base = (long long)blockIdx.y * outer_stride + c0;
    valid = (int)((npen - c0) < 16 ? (npen - c0) : 16);
  }
  const float* st_src[3] = {io.mult, io.mult2, io.accumulate ? io.out : nullptr};
  const bool full = vec && valid == 16;
#pragma unroll
  for (int fi = 0; fi < 3; ++fi) {
    const float* g = st_src[fi];
    if (!g) continue;
    float* d = stg + fi * FIELD;
    if (ROWS) {
      if (full) {
        for (int c = t; c < 16 * (L / 4); c += 256) {
          const int r = c >> 6, q = c & 63;
          cpa16(d + r * PITCH + 4 * q, g + base + (long long)r * L + 4 * q);
        }
      } else {
        for (int e = t; e < valid * L; e += 256) {
          const int r = e >> 8, n = e & 255;
          cpa_elem<float>(d + r * PITCH + n, g + base + (long long)r * L + n);
        }
      }
    } else {
      if (full) {
        for (int c = t; c < L * 4; c += 256) {
          const int n = c >> 2, q = c & 3;
          cpa16(d + n * 16 + 4 * q, g + base + (long long)n * S + 4 * q);
        }
      } else {
        for (int e = t; e < L * 16; e += 256) {
          const int n = e >> 4, c = e & 15;
          if (c < valid) cpa_elem<float>(d + n * 16 + c, g + base + (long long)n * S + c);
        }
      }
    }
  }
  cpa_commit();
  load_tw256<float>(tw, twg);
  const bool v0 = p < valid;
  const long long off = base + (ROWS ? (long long)p * L + x : p + (long long)x * S);
  const long long st16 = ROWS ? 16 : 16 * S;
  float2 a[16];
  {
    const float* fp = io.f + off;
    const float* f2p = io.f2 + off;
#pragma unroll
    for (int m = 0; m < 16; ++m) {
      a[m] = v0 ? make_float2(fp[0], f2p[0]) : make_float2(0.f, 0.f);
      fp += st16;
      f2p += st16;
    }
  }
  __syncthreads();  // twiddle table
  reg256_deriv_split(a, tw, xr + p * kX16P, x);
  cpa_wait<0>();
  __syncthreads();
  if (!v0) return;
  const float inv = 1.f / 256.f;
  long long e = off;
#pragma unroll
  for (int n2 = 0; n2 < 16; ++n2, e += st16) {
    const int n = x + 16 * n2;
    const int i = ROWS ? p * PITCH + n : n * 16 + p;
    float w1 = io.coef * (a[n2].x * inv);
    if (io.mult) w1 *= stg[i];
    if (io.accumulate) w1 += stg[2 * FIELD + i];
    float w2 = io.coef2 * (a[n2].y * inv);
    if (io.mult2) w2 *= stg[FIELD + i];
    io.out[e] = w2 + w1;
  }
}

// ---- real-to-complex FFT of row pairs ---------------------------------------------------------
template <typename T, int NC>
__global__ void __launch_bounds__(kThreads)
k_r2c_rows(const T* __restrict__ f, cx<T>* __restrict__ fh, long long rows, int Lr, int Lh, int B,
           int ld, FftPlan plan, const cx<T>* __restrict__ twg, int vec) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int L = NC > 0 ? NC : Lr;
  DerivSmem<T> sm(smem_raw, L, B, ld);
  const long long row0 = (long long)blockIdx.x * 2 * B;
  const int nrows = (int)((rows - row0) < 2 * B ? (rows - row0) : 2 * B);
  stage_contig<T>(sm.raw, f + row0 * L, nrows * L, nrows == 2 * B && vec);
  cpa_commit();
  load_tw<T>(sm.tw, twg, L);
  cpa_wait<0>();
  __syncthreads();
  for (int idx = threadIdx.x; idx < B * L; idx += blockDim.x) {
    const int p = idx / L, j = idx - p * L;
    const T va = (2 * p < nrows) ? sm.raw[(2 * p) * L + j] : T(0);
    const T vb = (2 * p + 1 < nrows) ? sm.raw[(2 * p + 1) * L + j] : T(0);
    sm.a[p * ld + pd(j)] = mk<T>(va, vb);
  }
  __syncthreads();
  const cx<T>* r = run_fft<T, NC>(sm.a, sm.b, L, B, ld, plan, sm.tw);
  StridedQR qr(threadIdx.x, Lh);
  for (int idx = threadIdx.x; idx < 2 * B * Lh; idx += blockDim.x, qr.next()) {
    const int rr = qr.q, k = qr.r;
    if (rr >= nrows) continue;
    const int p = rr >> 1;
    const cx<T> zk = r[p * ld + pd(k)];
    const cx<T> zm = cconj(r[p * ld + pd(k == 0 ? 0 : L - k)]);
    // row 2p: A_k = (Z_k + conj Z_-k) / 2;  row 2p+1: B_k = (Z_k - conj Z_-k) / (2 i)
    fh[(row0 + rr) * Lh + k] = (rr & 1) ? cscale(cmul_negi(csub(zk, zm)), T(0.5)) : cscale(cadd(zk, zm), T(0.5));
  }
}

// ---- complex-to-real inverse FFT of row pairs (normalised by `scale`) --------------------------
template <typename T, int NC>
__global__ void __launch_bounds__(kThreads)
k_c2r_rows(const cx<T>* __restrict__ fh, T* __restrict__ f, long long rows, int Lr, int Lh, int B,
           int ld, FftPlan plan, const cx<T>* __restrict__ twg, T scale, int vec) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int L = NC > 0 ? NC : Lr;
  DerivSmem<T> sm(smem_raw, L, B, ld);
  const long long row0 = (long long)blockIdx.x * 2 * B;
  const int nrows = (int)((rows - row0) < 2 * B ? (rows - row0) : 2 * B);
  // the 2B x Lh complex block is contiguous; it is staged in the raw multiplier area
  cx<T>* stg = reinterpret_cast<cx<T>*>(sm.mult);
  stage_contig<T>(reinterpret_cast<T*>(stg), reinterpret_cast<const T*>(fh + row0 * Lh), 2 * nrows * Lh,
                  nrows == 2 * B && vec);
  cpa_commit();
  load_tw<T>(sm.tw, twg, L);
  cpa_wait<0>();
  __syncthreads();
  // Z_k = A_k + i B_k (k < Lh) and Z_{L-k} = conj(A_k) + i conj(B_k); store conj(Z) in `a`.
  StridedQR qr(threadIdx.x, Lh);
  for (int idx = threadIdx.x; idx < B * Lh; idx += blockDim.x, qr.next()) {
    const int p = qr.q, k = qr.r;
    const cx<T> A = (2 * p < nrows) ? stg[(2 * p) * Lh + k] : mk<T>(T(0), T(0));
    const cx<T> Bv = (2 * p + 1 < nrows) ? stg[(2 * p + 1) * Lh + k] : mk<T>(T(0), T(0));
    sm.a[p * ld + pd(k)] = cconj(mk<T>(A.x - Bv.y, A.y + Bv.x));
    if (k >= 1 && L - k >= Lh) sm.a[p * ld + pd(L - k)] = cconj(mk<T>(A.x + Bv.y, -A.y + Bv.x));
  }
  __syncthreads();
  const cx<T>* r = run_fft<T, NC, 8>(sm.a, sm.b, L, B, ld, plan, sm.tw);
  for (int idx = threadIdx.x; idx < nrows * L; idx += blockDim.x) {
    const int rr = idx / L, j = idx - rr * L;
    const cx<T> z = r[(rr >> 1) * ld + pd(j)];
    f[row0 * L + idx] = ((rr & 1) ? -z.y : z.x) * scale;
  }
}

// ---- complex FFT along a strided axis of the half spectrum, in place ---------------------------
template <typename T> __device__ __forceinline__ void cpa_cx(cx<T>* sdst, const cx<T>* gsrc) {
  if constexpr (sizeof(T) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"((unsigned)__cvta_generic_to_shared(sdst)),
                 "l"(gsrc));
  else
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"((unsigned)__cvta_generic_to_shared(sdst)),
                 "l"(gsrc));
}

template <typename T, int NC>
__global__ void __launch_bounds__(kThreads)
k_fft_cols(cx<T>* __restrict__ fh, int Lr, long long S, long long outer_stride, int nx, int B, int ld,
           FftPlan plan, const cx<T>* __restrict__ twg, int inverse, T scale) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int L = NC > 0 ? NC : Lr;
  cx<T>* tw = reinterpret_cast<cx<T>*>(smem_raw);
  cx<T>* a = tw + ((L + 1) & ~1);
  cx<T>* b = a + (((size_t)B * ld + 1) & ~(size_t)1);
  const int x0 = blockIdx.x * B;
  const long long base = (long long)blockIdx.y * outer_stride + x0;
  const int valid = (nx - x0) < B ? (nx - x0) : B;
  // stage the tile as b[j * B + p]
  {
    StridedQR qr(threadIdx.x, B);
    for (int idx = threadIdx.x; idx < B * L; idx += blockDim.x, qr.next())
      if (qr.r < valid) cpa_cx<T>(b + idx, fh + base + qr.q * S + qr.r);
  }
  cpa_commit();
  load_tw<T>(tw, twg, L);
  cpa_wait<0>();
  __syncthreads();
  StridedQR qa(threadIdx.x, B);
  for (int idx = threadIdx.x; idx < B * L; idx += blockDim.x, qa.next()) {
    const int j = qa.q, p = qa.r;
    cx<T> z = (p < valid) ? b[idx] : mk<T>(T(0), T(0));
    if (inverse) z = cconj(z);
    a[p * ld + pd(j)] = z;
  }
  __syncthreads();
  const cx<T>* r = run_fft<T, NC>(a, b, L, B, ld, plan, tw);
  StridedQR qb(threadIdx.x, B);
  for (int idx = threadIdx.x; idx < B * L; idx += blockDim.x, qb.next()) {
    const int j = qb.q, p = qb.r;
    if (p >= valid) continue;
    cx<T> z = r[p * ld + pd(j)];
    if (inverse) z = cscale(cconj(z), scale);
    fh[base + j * S + p] = z;
  }
}

// pencils per CTA: about 4096 complex fp32 (2048 fp64) values per buffer
template <typename T> int batch_for(int L) {
  const int target = sizeof(T) == 4 ? 4096 : 2048;
  int B = target / L;
  return B < 1 ? 1 : B;
}
// pitch of one pencil in a work buffer: room for the padded index of element L - 1, made odd so that
// the same element of consecutive pencils falls in different banks
inline int lead_dim(int L) {
  const int ld = L + (L >> PS) + 1;
  return (ld % 2 == 0) ? ld + 1 : ld;
}
template <typename T> size_t smem_bytes(int L, int B) {
  const size_t twn = ((size_t)L + 1) & ~(size_t)1, bufn = ((size_t)B * lead_dim(L) + 1) & ~(size_t)1;
  return sizeof(cx<T>) * (twn + 2 * bufn);
}

// Calls f(std::integral_constant<int, NC>) with NC = L for the FP32 lengths that have a compile-time
// plan, else NC = 0 (runtime plan).
template <typename T, typename F> cudaError_t with_nc(int L, F&& f) {
  if constexpr (sizeof(T) == 4) {
    switch (L) {
      case 64: return f(std::integral_constant<int, 64>());
      case 96: return f(std::integral_constant<int, 96>());
      case 128: return f(std::integral_constant<int, 128>());
      case 160: return f(std::integral_constant<int, 160>());
      case 192: return f(std::integral_constant<int, 192>());
      case 256: return f(std::integral_constant<int, 256>());
      default: break;
    }
  }
  return f(std::integral_constant<int, 0>());
}

// Opt a kernel into large dynamic shared memory. The limit is a process-wide property of the kernel,
// so it is always raised to the device's opt-in maximum (never to one launch's size): concurrent
// host threads launching the same kernel with different sizes cannot lower it under each other.
inline int smem_optin_max() {
  static std::once_flag once;
  static int bytes = 48 * 1024;
  std::call_once(once, [] {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) == cudaSuccess && v > 0)
      bytes = v;
  });
  return bytes;
}
template <typename K> cudaError_t allow_smem(K kernel, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  if (bytes > (size_t)smem_optin_max()) return cudaErrorInvalidValue;
  // once per kernel: later launches (and launches recorded into a CUDA graph) make no attribute call
  static std::mutex mu;
  static std::unordered_set<const void*> done;
  std::lock_guard<std::mutex> lk(mu);
  if (done.count(reinterpret_cast<const void*>(kernel))) return cudaSuccess;
  const cudaError_t e =
      cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_optin_max());
  if (e == cudaSuccess) done.insert(reinterpret_cast<const void*>(kernel));
  return e;
}

}  // namespace

// pencils per CTA of the derivative kernels: 2048 complex fp32 (1024 fp64) values per buffer
template <typename T> int deriv_batch(int L) {
  const int target = sizeof(T) == 4 ? 2048 : 1024;
  int B = target / L;
  return B < 1 ? 1 : B;
}
template <typename T> size_t deriv_smem_bytes(int L, int B) {
  // twiddles + two complex buffers (each padded to an even count) + raw multiplier and accumulator
  // blocks (2B x L reals each)
  const size_t twn = ((size_t)L + 1) & ~(size_t)1, bufn = ((size_t)B * lead_dim(L) + 1) & ~(size_t)1;
  return sizeof(cx<T>) * (twn + 2 * bufn) + 2 * sizeof(T) * 2 * (size_t)B * L;
}

template <typename T, bool PAIR>
static cudaError_t deriv_pass(const Grid& g, const FftTables<T>& ft, int axis, const DerivIO<T>& io, cudaStream_t st) {
  const int L = g.n[axis];
  if (L == 1) {  // a singleton axis carries only k = 0: the derivative is zero
    if (io.accumulate) return cudaSuccess;
    return cudaMemsetAsync(io.out, 0, sizeof(T) * g.nvox, st);
  }
  if constexpr (std::is_same<T, float>::value && PAIR) {
    if (L == kRegFftLen) {  // register-resident transform with staged operands (k_deriv_pair256s)
      const auto al = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
      const bool ptrs16 = (!io.mult || al(io.mult)) && (!io.mult2 || al(io.mult2)) && (!io.accumulate || al(io.out));
      if (axis == 2) {
        const long long rows = (long long)g.n[0] * g.n[1];
        auto kern = k_deriv_pair256s<true>;
        constexpr size_t sm = Reg256S<true>::bytes();
        cudaError_t e = allow_smem(kern, sm);
        if (e != cudaSuccess) return e;
        note_launches(1);
        kern<<<(unsigned)((rows + 15) / 16), 256, sm, st>>>(io, rows, 1, 0, ft.tw[2], ptrs16 ? 1 : 0);
        return cudaGetLastError();
      }
      const int nx = g.n[2];
      long long S, outer_stride;
      int outer;
      if (axis == 1) {
        S = nx;
        outer = g.n[0];
        outer_stride = (long long)g.n[1] * nx;
      } else {
        S = (long long)g.n[1] * nx;
        outer = g.n[1];
        outer_stride = nx;
      }
      auto kern = k_deriv_pair256s<false>;
      constexpr size_t sm = Reg256S<false>::bytes();
      cudaError_t e = allow_smem(kern, sm);
      if (e != cudaSuccess) return e;
      note_launches(1);
      // 16-byte copies of column segments: rows of whole chunks (nx a multiple of 4)
      const int vec = (ptrs16 && nx % 4 == 0) ? 1 : 0;
      kern<<<dim3((unsigned)((nx + 15) / 16), (unsigned)outer), 256, sm, st>>>(io, nx, S, outer_stride, ft.tw[axis],
                                                                                 vec);
      return cudaGetLastError();
    }
  }
  if (L == kRegFftLen) {  // register-resident transform (k_deriv_reg256: FP64, and the one-field FP32 passes)
    const size_t sm = sizeof(cx<T>) * (256 + 16 * kX16P);
    constexpr int rp = PAIR ? 1 : 2;
    if (axis == 2) {
      const long long rows = (long long)g.n[0] * g.n[1];
      auto kern = k_deriv_reg256<T, PAIR, true>;
      cudaError_t e = allow_smem(kern, sm);
      if (e != cudaSuccess) return e;
      note_launches(1);
      kern<<<(unsigned)((rows + 16 * rp - 1) / (16 * rp)), 256, sm, st>>>(io, rows, 1, 0, ft.tw[2]);
      return cudaGetLastError();
    }
    const int nx = g.n[2];
    long long S, outer_stride;
    int outer;
    if (axis == 1) {
      S = nx;
      outer = g.n[0];
      outer_stride = (long long)g.n[1] * nx;
    } else {
      S = (long long)g.n[1] * nx;
      outer = g.n[1];
      outer_stride = nx;
    }
    auto kern = k_deriv_reg256<T, PAIR, false>;
    cudaError_t e = allow_smem(kern, sm);
    if (e != cudaSuccess) return e;
    note_launches(1);
    kern<<<dim3((unsigned)((nx + 16 * rp - 1) / (16 * rp)), (unsigned)outer), 256, sm, st>>>(io, nx, S, outer_stride,
                                                                                            ft.tw[axis]);
    return cudaGetLastError();
  }
  const int tuned = PAIR ? ft.pair_pencils[axis] : ft.deriv_pencils[axis];
  int B = tuned > 0 ? tuned : deriv_batch<T>(L);
  const int ld = lead_dim(L);
  const auto al = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
  const bool ptrs16 = al(io.f) && al(io.out) && (!io.mult || al(io.mult)) && (!PAIR || al(io.f2)) &&
                      (!PAIR || !io.mult2 || al(io.mult2));
  constexpr int per = 16 / sizeof(T);
  constexpr int rpc = PAIR ? 1 : 2;  // real pencils of one field per complex pencil
  if (axis == 2) {
    const long long rows = (long long)g.n[0] * g.n[1];
    const long long most = (rows + rpc - 1) / rpc;
    if (B > most) B = (int)most;
    const size_t sm = deriv_smem_bytes<T>(L, B);
    const long long grid = (rows + (long long)rpc * B - 1) / ((long long)rpc * B);
    const int vec = (ptrs16 && (L % per) == 0) ? 1 : 0;
    return with_nc<T>(L, [&](auto nc) {
      constexpr int NC = decltype(nc)::value;
      cudaError_t e = allow_smem(k_deriv_rows<T, NC, PAIR>, sm);
      if (e != cudaSuccess) return e;
      note_launches(1);
      k_deriv_rows<T, NC, PAIR><<<(unsigned)grid, kThreads, sm, st>>>(io, rows, L, B, ld, ft.plan[2], ft.tw[2], vec);
      return cudaGetLastError();
    });
  }
  const int nx = g.n[2];
  if (rpc * B > nx) B = (nx + rpc - 1) / rpc;
  const int W = rpc * B;
  const size_t sm = deriv_smem_bytes<T>(L, B);
  long long S, outer_stride;
  int outer;
  if (axis == 1) {
    S = nx;
    outer = g.n[0];
    outer_stride = (long long)g.n[1] * nx;
  } else {
    S = (long long)g.n[1] * nx;
    outer = g.n[1];
    outer_stride = nx;
  }
  // 16-byte chunks need whole chunks per tile row and 16-byte aligned row starts
  const int vec = (ptrs16 && W % per == 0 && (nx % per) == 0) ? 1 : 0;
  dim3 grid((nx + W - 1) / W, outer);
  return with_nc<T>(L, [&](auto nc) {
    constexpr int NC = decltype(nc)::value;
    cudaError_t e = allow_smem(k_deriv_cols<T, NC, PAIR>, sm);
    if (e != cudaSuccess) return e;
    note_launches(1);
    k_deriv_cols<T, NC, PAIR><<<grid, kThreads, sm, st>>>(io, L, S, outer_stride, nx, B, ld, ft.plan[axis],
                                                           ft.tw[axis], vec);
    return cudaGetLastError();
  });
}

template <typename T>
cudaError_t launch_deriv(const Grid& g, const FftTables<T>& ft, int axis, const T* f, const T* mult,
                         T* out, T coef, bool accumulate, cudaStream_t st) {
  const DerivIO<T> io{f, mult, nullptr, nullptr, out, coef, T(0), accumulate ? 1 : 0};
  return deriv_pass<T, false>(g, ft, axis, io, st);
}

template <typename T>
cudaError_t launch_deriv_pair(const Grid& g, const FftTables<T>& ft, int axis, const T* f, const T* mult, T coef,
                              const T* f2, const T* mult2, T coef2, T* out, bool accumulate, cudaStream_t st) {
  const DerivIO<T> io{f, mult, f2, mult2, out, coef, coef2, accumulate ? 1 : 0};
  return deriv_pass<T, true>(g, ft, axis, io, st);
}

// Complex transform of 16 columns per CTA along a strided 256-point axis, in registers (the four-step
// form above, forward only): thread (p, x) loads x[x + 16 m] of column p, applies the DFT16 over m and
// the twiddles W256^(x k2), one exchange gives it the values over q for k2 = x, and the DFT16 over q
// leaves X[x + 16 k1] in a[k1], which it stores where it loaded. The inverse conjugates on the way in
// and on the way out (times scale), as k_fft_cols does. Columns past nx are zero and not stored.
template <typename T, bool INV>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 2)
k_fft_cols_reg256(cx<T>* __restrict__ fh, long long S, long long outer_stride, int nx,
                  const cx<T>* __restrict__ twg, T scale) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* tw = reinterpret_cast<cx<T>*>(smem_raw);  // W256^(a b) at b * 16 + a (load_tw256)
  cx<T>* xb = tw + 256;                             // exchange buffer, kX16P per column
  load_tw256<T>(tw, twg);
  const int t = threadIdx.x, p = t & 15, x = t >> 4;
  const int c0 = blockIdx.x * 16;
  const bool v0 = c0 + p < nx;
  const long long off = (long long)blockIdx.y * outer_stride + c0 + p + (long long)x * S;
  const long long st16 = 16 * S;
  cx<T> a[16];
  {
    const cx<T>* fp = fh + off;
#pragma unroll
    for (int m = 0; m < 16; ++m, fp += st16) {
      cx<T> z = v0 ? fp[0] : mk<T>(T(0), T(0));
      if (INV) z = cconj(z);
      a[m] = z;
    }
  }
  __syncthreads();  // twiddle table
  dft16<T>(a);
#pragma unroll
  for (int k2 = 1; k2 < 16; ++k2) a[k2] = cmul(a[k2], tw[k2 * 16 + x]);
  cx<T>* xp = xb + p * kX16P;
#pragma unroll
  for (int k2 = 0; k2 < 16; ++k2) xp[k2 * 17 + x] = a[k2];
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 16; ++q) a[q] = xp[x * 17 + q];  // thread holds k2 = x over q
  dft16<T>(a);                                          // a[k1] = X[x + 16 k1]
  if (!v0) return;
  cx<T>* op = fh + off;
#pragma unroll
  for (int k1 = 0; k1 < 16; ++k1, op += st16) op[0] = INV ? cscale(cconj(a[k1]), scale) : a[k1];
}

// Row passes of the 3D real FFT for 256-point rows, in registers: 16 complex pencils per CTA, pencil p
// packing rows 2p and 2p + 1 of the tile as real and imaginary parts, transformed as 16 x 16 with one
// exchange (thread (p, x) holds the values at x + 16 m before and the bins x + 16 k1 after the
// transform). The half spectra of the two rows, A_k = (Z_k + conj Z_{256-k}) / 2 and
// B_k = (Z_k - conj Z_{256-k}) / (2 i), need bin 256 - k, which thread (p, (16 - x) mod 16) of the same
// half-warp holds (in a[15 - k1], or a[(16 - k1) mod 16] when x = 0): one shuffle per bin brings it.
template <typename T>
__device__ __forceinline__ void reg256_forward(cx<T>* a, const cx<T>* tw, cx<T>* xp, int x) {
  dft16<T>(a);
#pragma unroll
  for (int k2 = 1; k2 < 16; ++k2) a[k2] = cmul(a[k2], tw[k2 * 16 + x]);
#pragma unroll
  for (int k2 = 0; k2 < 16; ++k2) xp[k2 * 17 + x] = a[k2];
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 16; ++q) a[q] = xp[x * 17 + q];  // thread holds k2 = x over q
  dft16<T>(a);                                          // a[k1] = X[x + 16 k1]
}

template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 2)
k_r2c_rows_reg256(const T* __restrict__ f, cx<T>* __restrict__ fh, long long rows, const cx<T>* __restrict__ twg) {
  constexpr int L = 256, LH = 129;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* tw = reinterpret_cast<cx<T>*>(smem_raw);
  cx<T>* xb = tw + L;
  load_tw256<T>(tw, twg);
  const int t = threadIdx.x, p = t >> 4, x = t & 15;
  const long long r0 = (long long)blockIdx.x * 32 + 2 * p;
  const bool va = r0 < rows, vb = r0 + 1 < rows;
  cx<T> a[16];
  {
    const T* fa = f + r0 * L + x;
#pragma unroll
    for (int m = 0; m < 16; ++m) a[m] = mk<T>(va ? fa[16 * m] : T(0), vb ? fa[L + 16 * m] : T(0));
  }
  __syncthreads();  // twiddle table
  reg256_forward<T>(a, tw, xb + p * kX16P, x);
  const int lane = t & 31, partner = (lane & 16) | ((16 - x) & 15);
  cx<T> r[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    r[i].x = __shfl_sync(0xffffffffu, a[i].x, partner);
    r[i].y = __shfl_sync(0xffffffffu, a[i].y, partner);
  }
  cx<T>* ha = fh + r0 * LH + x;
#pragma unroll
  for (int k1 = 0; k1 <= 8; ++k1) {
    if (k1 == 8 && x != 0) break;  // bins x + 16 k1 <= 128
    const cx<T> zk = a[k1];
    const cx<T> zm = cconj(x != 0 ? r[15 - k1] : r[(16 - k1) & 15]);
    if (va) ha[16 * k1] = cscale(cadd(zk, zm), T(0.5));
    if (vb) ha[LH + 16 * k1] = cscale(cmul_negi(csub(zk, zm)), T(0.5));
  }
}

// The inverse: Z_k = A_k + i B_k for k <= 128 and Z_{256-k} = conj A_k + i conj B_k, transformed
// through conjugation; row 2p is the real part, row 2p + 1 the imaginary part (times scale).
template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 2)
k_c2r_rows_reg256(const cx<T>* __restrict__ fh, T* __restrict__ f, long long rows, const cx<T>* __restrict__ twg,
                  T scale) {
  constexpr int L = 256, LH = 129;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* tw = reinterpret_cast<cx<T>*>(smem_raw);
  cx<T>* xb = tw + L;
  load_tw256<T>(tw, twg);
  const int t = threadIdx.x, p = t >> 4, x = t & 15;
  const long long r0 = (long long)blockIdx.x * 32 + 2 * p;
  const bool va = r0 < rows, vb = r0 + 1 < rows;
  const cx<T>* ha = fh + r0 * LH;
  const cx<T> zero = mk<T>(T(0), T(0));
  cx<T> a[16];
#pragma unroll
  for (int m = 0; m < 16; ++m) {
    const int n = x + 16 * m;
    const bool direct = n <= 128;
    const int k = direct ? n : L - n;
    const cx<T> A = va ? ha[k] : zero, Bv = vb ? ha[LH + k] : zero;
    const cx<T> z = direct ? mk<T>(A.x - Bv.y, A.y + Bv.x) : mk<T>(A.x + Bv.y, -A.y + Bv.x);
    a[m] = cconj(z);
  }
  __syncthreads();  // twiddle table
  reg256_forward<T>(a, tw, xb + p * kX16P, x);
  T* fa = f + r0 * L + x;
#pragma unroll
  for (int k1 = 0; k1 < 16; ++k1) {
    if (va) fa[16 * k1] = a[k1].x * scale;
    if (vb) fa[L + 16 * k1] = -a[k1].y * scale;
  }
}

template <typename T>
static cudaError_t launch_cols(const Grid& g, const FftTables<T>& ft, int axis, cx<T>* fh, int inverse,
                               cudaStream_t st) {
  const int L = g.n[axis];
  if (L == 1) return cudaSuccess;
  const int nx = g.n2h;
  int B = batch_for<T>(L);
  if (B > nx) B = nx;
  const int ld = lead_dim(L);
  const size_t sm = smem_bytes<T>(L, B);
  long long S, outer_stride;
  int outer;
  if (axis == 1) {
    S = nx;
    outer = g.n[0];
    outer_stride = (long long)g.n[1] * nx;
  } else {
    S = (long long)g.n[1] * nx;
    outer = g.n[1];
    outer_stride = nx;
  }
  if (L == kRegFftLen) {  // register-resident transform: 16 columns per CTA
    auto kern = inverse ? k_fft_cols_reg256<T, true> : k_fft_cols_reg256<T, false>;
    const size_t smr = sizeof(cx<T>) * (256 + 16 * kX16P);
    cudaError_t e = allow_smem(kern, smr);
    if (e != cudaSuccess) return e;
    note_launches(1);
    kern<<<dim3((nx + 15) / 16, outer), 256, smr, st>>>(fh, S, outer_stride, nx, ft.tw[axis], T(1) / T(L));
    return cudaGetLastError();
  }
  dim3 grid((nx + B - 1) / B, outer);
  return with_nc<T>(L, [&](auto nc) {
    constexpr int NC = decltype(nc)::value;
    cudaError_t e = allow_smem(k_fft_cols<T, NC>, sm);
    if (e != cudaSuccess) return e;
    note_launches(1);
    k_fft_cols<T, NC><<<grid, kThreads, sm, st>>>(fh, L, S, outer_stride, nx, B, ld, ft.plan[axis], ft.tw[axis],
                                                   inverse, T(1) / T(L));
    return cudaGetLastError();
  });
}

template <typename T>
cudaError_t launch_r2c(const Grid& g, const FftTables<T>& ft, const T* f, cx<T>* fh, cudaStream_t st) {
  const int L = g.n[2];
  const long long rows = (long long)g.n[0] * g.n[1];
  if (L == kRegFftLen) {  // register-resident row pass: 32 rows per CTA
    auto kern = k_r2c_rows_reg256<T>;
    const size_t smr = sizeof(cx<T>) * (256 + 16 * kX16P);
    cudaError_t e = allow_smem(kern, smr);
    if (e != cudaSuccess) return e;
    note_launches(1);
    kern<<<(unsigned)((rows + 31) / 32), 256, smr, st>>>(f, fh, rows, ft.tw[2]);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = launch_cols<T>(g, ft, 1, fh, 0, st)) != cudaSuccess) return e;
    return launch_cols<T>(g, ft, 0, fh, 0, st);
  }
  int B = batch_for<T>(L);
  if (B > (rows + 1) / 2) B = (int)((rows + 1) / 2);
  const int ld = lead_dim(L);
  const size_t sm = smem_bytes<T>(L, B);
  const long long grid = (rows + 2LL * B - 1) / (2LL * B);
  constexpr int per = 16 / sizeof(T);
  const int vec = ((reinterpret_cast<uintptr_t>(f) & 15u) == 0 && L % per == 0) ? 1 : 0;
  cudaError_t e = with_nc<T>(L, [&](auto nc) {
    constexpr int NC = decltype(nc)::value;
    cudaError_t e2 = allow_smem(k_r2c_rows<T, NC>, sm);
    if (e2 != cudaSuccess) return e2;
    note_launches(1);
    k_r2c_rows<T, NC><<<(unsigned)grid, kThreads, sm, st>>>(f, fh, rows, L, g.n2h, B, ld, ft.plan[2], ft.tw[2],
                                                             vec);
    return cudaGetLastError();
  });
  if (e != cudaSuccess) return e;
  if ((e = launch_cols<T>(g, ft, 1, fh, 0, st)) != cudaSuccess) return e;
  return launch_cols<T>(g, ft, 0, fh, 0, st);
}

template <typename T>
cudaError_t launch_c2r(const Grid& g, const FftTables<T>& ft, cx<T>* fh, T* f, cudaStream_t st) {
  cudaError_t e;
  if ((e = launch_cols<T>(g, ft, 0, fh, 1, st)) != cudaSuccess) return e;
  if ((e = launch_cols<T>(g, ft, 1, fh, 1, st)) != cudaSuccess) return e;
  const int L = g.n[2];
  const long long rows = (long long)g.n[0] * g.n[1];
  if (L == kRegFftLen) {  // register-resident row pass: 32 rows per CTA
    auto kern = k_c2r_rows_reg256<T>;
    const size_t smr = sizeof(cx<T>) * (256 + 16 * kX16P);
    if ((e = allow_smem(kern, smr)) != cudaSuccess) return e;
    note_launches(1);
    kern<<<(unsigned)((rows + 31) / 32), 256, smr, st>>>(fh, f, rows, ft.tw[2], T(1) / T(L));
    return cudaGetLastError();
  }
  int B = deriv_batch<T>(L);  // the staged half-spectrum block uses the multiplier/accumulator area
  if (B > (rows + 1) / 2) B = (int)((rows + 1) / 2);
  const int ld = lead_dim(L);
  const size_t sm = deriv_smem_bytes<T>(L, B);
  const long long grid = (rows + 2LL * B - 1) / (2LL * B);
  const int vec = (reinterpret_cast<uintptr_t>(fh) & 15u) == 0 ? 1 : 0;
  return with_nc<T>(L, [&](auto nc) {
    constexpr int NC = decltype(nc)::value;
    cudaError_t e2 = allow_smem(k_c2r_rows<T, NC>, sm);
    if (e2 != cudaSuccess) return e2;
    note_launches(1);
    k_c2r_rows<T, NC><<<(unsigned)grid, kThreads, sm, st>>>(fh, f, rows, L, g.n2h, B, ld, ft.plan[2], ft.tw[2],
                                                             T(1) / T(L), vec);
    return cudaGetLastError();
  });
}

template <typename T> int deriv_default_pencils(int L) { return deriv_batch<T>(L); }
template <typename T> bool deriv_pencils_fit(int L, int B) {
  return B >= 1 && deriv_smem_bytes<T>(L, B) <= (size_t)smem_optin_max();
}

#define GA_INST(T)                                                                                  \
  template int deriv_default_pencils<T>(int);                                                       \
  template bool deriv_pencils_fit<T>(int, int);                                                     \
  template cudaError_t launch_deriv<T>(const Grid&, const FftTables<T>&, int, const T*, const T*, T*, T, \
                                       bool, cudaStream_t);                                          \
  template cudaError_t launch_deriv_pair<T>(const Grid&, const FftTables<T>&, int, const T*, const T*, T,  \
                                            const T*, const T*, T, T*, bool, cudaStream_t);          \
  template cudaError_t launch_r2c<T>(const Grid&, const FftTables<T>&, const T*, cx<T>*, cudaStream_t); \
  template cudaError_t launch_c2r<T>(const Grid&, const FftTables<T>&, cx<T>*, T*, cudaStream_t);
GA_INST(float)
GA_INST(double)
#undef GA_INST

}  // namespace ga
