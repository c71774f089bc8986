// Tiled FP32 semi-Lagrangian step for 3D grids (Sec. 2.2; same arithmetic as sl_kernels.cu).
//
// A CTA owns a brick of 32 x 8 x 8 voxels (x contiguous). It stages the brick plus a periodic halo
// (4 cells below / 4 above in x, 3 / 3 in y and z) of the transported field into shared memory with
// 16-byte cp.async copies (and mu for the two-field steps). Each thread owns a column of 8 voxels
// along z and interpolates them one by one: a departure point whose integer offset lies in [-2, 1]
// on every axis reads its 64 taps from shared memory (the product f * mu is formed tap by tap); any
// other departure point reads the field from global memory, so every displacement is handled
// exactly.
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>

#include "kernels.h"

namespace ga {

namespace {

constexpr int BX = 32, BY = 8, BZ = 8, H = 2;
constexpr int TY = BY + 2 * H + 2, TZ = BZ + 2 * H + 2;  // 14, 14 (x extent: TXA below)

__device__ __forceinline__ int wrap_any(int a, int n) {
  a %= n;
  return a < 0 ? a + n : a;
}

__device__ __forceinline__ void lagrange4(float t, float* w) {
  const float tp1 = t + 1.f, tm1 = t - 1.f, tm2 = t - 2.f;
  const float sixth = 1.f / 6.f;
  w[0] = -t * tm1 * tm2 * sixth;
  w[1] = tp1 * tm1 * tm2 * 0.5f;
  w[2] = -tp1 * t * tm2 * 0.5f;
  w[3] = tp1 * t * tm1 * sixth;
}

// 64-tap interpolation from global memory with periodic wrap (departure point outside the halo).
template <int NF>
__device__ __forceinline__ void gather_global(const float* __restrict__ f, const float* __restrict__ mu, int gz,
                                              int gy, int gx, float dz, float dy, float dx, int n0, int n1, int n2,
                                              float& P, float& S) {
  float wz[4], wy[4], wx[4];
  const float fz = floorf(dz), fy = floorf(dy), fx = floorf(dx);
  lagrange4(dz - fz, wz);
  lagrange4(dy - fy, wy);
  lagrange4(dx - fx, wx);
  const float lim = 1048576.f;
  const int iz = wrap_any(gz + (int)fminf(fmaxf(fz, -lim), lim) - 1, n0);
  const int iy = wrap_any(gy + (int)fminf(fmaxf(fy, -lim), lim) - 1, n1);
  const int ix = wrap_any(gx + (int)fminf(fmaxf(fx, -lim), lim) - 1, n2);
  int xs[4];
  for (int a = 0, x = ix; a < 4; ++a, x = (x + 1 == n2) ? 0 : x + 1) xs[a] = x;
  float acc = 0.f, accp = 0.f;
  for (int c = 0, z = iz; c < 4; ++c, z = (z + 1 == n0) ? 0 : z + 1) {
    float ay = 0.f, ayp = 0.f;
    for (int b = 0, y = iy; b < 4; ++b, y = (y + 1 == n1) ? 0 : y + 1) {
      const size_t row = ((size_t)z * n1 + y) * n2;
      float sx = 0.f, sxp = 0.f;
      for (int a = 0; a < 4; ++a) {
        const float v = __ldg(f + row + xs[a]);
        sx += wx[a] * v;
        if (NF == 2) sxp += wx[a] * v * __ldg(mu + row + xs[a]);
      }
      ay += wy[b] * sx;
      if (NF == 2) ayp += wy[b] * sxp;
    }
    acc += wz[c] * ay;
    if (NF == 2) accp += wz[c] * ayp;
  }
  P = acc;
  S = accp;
}

template <int MODE>
__device__ __forceinline__ void store_step(float* __restrict__ out, const float* __restrict__ mu, long long idx,
                                           float P, float S, float ht) {
  float o;
  if (MODE == 1) {
    const float m = mu[idx];
    o = P - 0.5f * ht * (S + m * (P - ht * S));
  } else if (MODE == 2) {
    const float m = mu[idx];
    o = P + 0.5f * ht * (S + m * (P + ht * S));
  } else {
    o = P;
  }
  out[idx] = o;
}

// ---- asynchronous global -> shared copies (LDGSTS) ----
__device__ __forceinline__ void cp_async16(float* sdst, const float* gsrc) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gsrc));
}
__device__ __forceinline__ void cp_async4(float* sdst, const float* gsrc) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gsrc));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }

// Staged tile: x extent TXA = 40 starting at bx*BX - 4 (16-byte aligned), y and z as before.
constexpr int TXA = 40, XOFF = 4;
constexpr int TILEA = TXA * TY * TZ;

struct BrickIdx {
  int bx, by, bz;
};
__device__ __forceinline__ BrickIdx brick_of(int b, int nbx, int nby) {
  BrickIdx r;
  r.bx = b % nbx;
  r.by = (b / nbx) % nby;
  r.bz = b / (nbx * nby);
  return r;
}

// Issue the copies of one brick's tile of `src` into `dst` (all threads of the CTA).
__device__ __forceinline__ void stage_async(float* dst, const float* __restrict__ src, const BrickIdx& bi, int n0,
                                            int n1, int n2, bool vec) {
  const int gx0 = bi.bx * BX - XOFF, gy0 = bi.by * BY - H - 1, gz0 = bi.bz * BZ - H - 1;
  if (vec) {  // 16-byte chunks: n2 % 4 == 0 and n2 >= TXA, so a chunk never straddles the wrap;
              // the launcher also requires n1 >= TY and n0 >= TZ so one conditional shift wraps y, z
    for (int c = threadIdx.x; c < TY * TZ * (TXA / 4); c += blockDim.x) {
      const int cx = c % (TXA / 4), row = c / (TXA / 4);
      const int ty = row % TY, tz = row / TY;
      int gy = gy0 + ty, gz = gz0 + tz;
      gy = gy < 0 ? gy + n1 : (gy >= n1 ? gy - n1 : gy);  // n1, n0 >= TY, TZ on this path
      gz = gz < 0 ? gz + n0 : (gz >= n0 ? gz - n0 : gz);
      int gx = gx0 + 4 * cx;
      gx = gx < 0 ? gx + n2 : (gx >= n2 ? gx - n2 : gx);
      cp_async16(dst + row * TXA + 4 * cx, src + ((size_t)gz * n1 + gy) * n2 + gx);
    }
  } else {
    for (int e = threadIdx.x; e < TILEA; e += blockDim.x) {
      const int tx = e % TXA, row = e / TXA;
      const int ty = row % TY, tz = row / TY;
      const int gy = wrap_any(gy0 + ty, n1), gz = wrap_any(gz0 + tz, n0);
      const int gx = wrap_any(gx0 + tx, n2);
      cp_async4(dst + e, src + ((size_t)gz * n1 + gy) * n2 + gx);
    }
  }
}

// MODE 0: advection state step          out = I[f](X-)
// MODE 1: continuity state step         out = P - ht/2 (S + mu (P - ht S)),  P = I[f], S = I[f mu]
// MODE 2: advection adjoint step        out = L + ht/2 (S + mu (L + ht S)),  L = I[f], S = I[f mu]
// MODE 3: continuity adjoint step       out = I[f](X+)
// One CTA per brick. The tile (and, for the two-field steps, mu) is copied asynchronously into
// shared memory; several CTAs per SM overlap one brick's copies with another's interpolation. Each
// thread interpolates its column of 8 voxels one voxel at a time: the 64 taps are read from shared
// memory at compile-time offsets from one base index per voxel.
template <int MODE>
__global__ void __launch_bounds__(256)
k_sl_tile(const float* __restrict__ f, const float* __restrict__ mu, const float* __restrict__ disp,
          float* __restrict__ out, int n0, int n1, int n2, float ht, int vec) {
  constexpr int NF = (MODE == 1 || MODE == 2) ? 2 : 1;  // staged fields: f (and mu)
  extern __shared__ __align__(16) float smem[];
  const float* sf = smem;
  const float* sm = smem + TILEA;
  const long long nv = (long long)n0 * n1 * n2;
  const int nbx = (n2 + BX - 1) / BX, nby = (n1 + BY - 1) / BY;
  const BrickIdx bi = brick_of(blockIdx.x, nbx, nby);
  stage_async(smem, f, bi, n0, n1, n2, vec != 0);
  if (NF == 2) stage_async(smem + TILEA, mu, bi, n0, n1, n2, vec != 0);
  cp_async_commit();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int gx = bi.bx * BX + lane, gy = bi.by * BY + warp;
  asm volatile("cp.async.wait_all;\n" ::);
  __syncthreads();
  if (gx >= n2 || gy >= n1) return;
  const int nz = min(BZ, n0 - bi.bz * BZ);
#pragma unroll 2
  for (int v = 0; v < nz; ++v) {
    const long long idx = ((long long)(bi.bz * BZ + v) * n1 + gy) * n2 + gx;
    const float vz = disp[idx], vy = disp[nv + idx], vx = disp[2 * nv + idx];
    const float fz = floorf(vz), fy = floorf(vy), fx = floorf(vx);
    float P = 0.f, S = 0.f;
    if (fz >= -H && fz <= H - 1 && fy >= -H && fy <= H - 1 && fx >= -H && fx <= H - 1) {
      float wz[4], wy[4], wx[4];
      lagrange4(vz - fz, wz);
      lagrange4(vy - fy, wy);
      lagrange4(vx - fx, wx);
      const int base = ((v + H + (int)fz) * TY + warp + H + (int)fy) * TXA + lane + XOFF - 1 + (int)fx;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        float ay = 0.f, ayp = 0.f;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const int o = base + (c * TY + b) * TXA;
          const float f0 = sf[o], f1 = sf[o + 1], f2 = sf[o + 2], f3 = sf[o + 3];
          ay += wy[b] * (wx[0] * f0 + wx[1] * f1 + wx[2] * f2 + wx[3] * f3);
          if (NF == 2)
            ayp += wy[b] * (wx[0] * f0 * sm[o] + wx[1] * f1 * sm[o + 1] + wx[2] * f2 * sm[o + 2] +
                            wx[3] * f3 * sm[o + 3]);
        }
        P += wz[c] * ay;
        if (NF == 2) S += wz[c] * ayp;
      }
    } else {
      gather_global<NF>(f, mu, bi.bz * BZ + v, gy, gx, vz, vy, vx, n0, n1, n2, P, S);
    }
    store_step<MODE>(out, mu, idx, P, S, ht);
  }
}

// RK2 departure points (displacements in cells) for 3D FP32 grids: X* = x -/+ h_t v(x), then
// X-/+ = x -/+ (h_t / 2)(v(x) + I[v](X*)). The three velocity components of the brick + halo are
// staged in shared memory; the three interpolants at X* share one stencil.
__global__ void __launch_bounds__(256, 2)
k_departure_tile(const float* __restrict__ v, float* __restrict__ xm, float* __restrict__ xp, int n0, int n1, int n2,
                 float ht, int both, int vec) {
  extern __shared__ __align__(16) float smem[];
  const long long nv = (long long)n0 * n1 * n2;
  const int nbx = (n2 + BX - 1) / BX, nby = (n1 + BY - 1) / BY;
  const BrickIdx bi = brick_of(blockIdx.x, nbx, nby);
  for (int c = 0; c < 3; ++c) stage_async(smem + c * TILEA, v + c * nv, bi, n0, n1, n2, vec != 0);
  cp_async_commit();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int gx = bi.bx * BX + lane, gy = bi.by * BY + warp;
  const float twopi = 6.283185307179586f;
  const float ih[3] = {(float)n0 / twopi, (float)n1 / twopi, (float)n2 / twopi};  // 1 / h_a
  asm volatile("cp.async.wait_all;\n" ::);
  __syncthreads();
  if (gx >= n2 || gy >= n1) return;
  const int nz = min(BZ, n0 - bi.bz * BZ);
#pragma unroll 1
  for (int vz = 0; vz < nz; ++vz) {
    const long long idx = ((long long)(bi.bz * BZ + vz) * n1 + gy) * n2 + gx;
    const int center = ((vz + H + 1) * TY + warp + H + 1) * TXA + lane + XOFF;
    float vc[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) vc[c] = smem[c * TILEA + center];
#pragma unroll 1
    for (int sg = 0; sg < (both ? 2 : 1); ++sg) {
      const float sign = sg == 0 ? 1.f : -1.f;
      float* o = sg == 0 ? xm : xp;
      const float dz = -sign * ht * vc[0] * ih[0], dy = -sign * ht * vc[1] * ih[1], dx = -sign * ht * vc[2] * ih[2];
      const float fz = floorf(dz), fy = floorf(dy), fx = floorf(dx);
      if (fz >= -H && fz <= H - 1 && fy >= -H && fy <= H - 1 && fx >= -H && fx <= H - 1) {
        float wz[4], wy[4], wx[4];
        lagrange4(dz - fz, wz);
        lagrange4(dy - fy, wy);
        lagrange4(dx - fx, wx);
        const int base = ((vz + H + (int)fz) * TY + warp + H + (int)fy) * TXA + lane + XOFF - 1 + (int)fx;
#pragma unroll 1
        for (int k = 0; k < 3; ++k) {  // one component at a time: the stencil weights are shared
          const float* t = smem + k * TILEA + base;
          float acc = 0.f;
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            float ay = 0.f;
#pragma unroll
            for (int b = 0; b < 4; ++b) {
              const float* r = t + (c * TY + b) * TXA;
              ay += wy[b] * (wx[0] * r[0] + wx[1] * r[1] + wx[2] * r[2] + wx[3] * r[3]);
            }
            acc += wz[c] * ay;
          }
          const float vk = k == 0 ? vc[0] : (k == 1 ? vc[1] : vc[2]);
          const float ihk = k == 0 ? ih[0] : (k == 1 ? ih[1] : ih[2]);
          o[k * nv + idx] = -sign * 0.5f * ht * (vk + acc) * ihk;
        }
      } else {
#pragma unroll 1
        for (int k = 0; k < 3; ++k) {
          float P, S;
          gather_global<1>(v + k * nv, nullptr, bi.bz * BZ + vz, gy, gx, dz, dy, dx, n0, n1, n2, P, S);
          const float vk = k == 0 ? vc[0] : (k == 1 ? vc[1] : vc[2]);
          const float ihk = k == 0 ? ih[0] : (k == 1 ? ih[1] : ih[2]);
          o[k * nv + idx] = -sign * 0.5f * ht * (vk + P) * ihk;
        }
      }
    }
  }
}

template <int MODE>
cudaError_t launch_mode(const Grid& g, const float* f, const float* mu, const float* disp, float* out, float ht,
                        cudaStream_t st) {
  constexpr int NF = (MODE == 1 || MODE == 2) ? 2 : 1;
  const size_t sm = sizeof(float) * TILEA * NF;  // two-field steps: TILEA float2 pairs
  static std::atomic<bool> attr{false};
  if (!attr.load()) {
    cudaError_t e = cudaFuncSetAttribute(k_sl_tile<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    attr.store(true);
  }
  const int nb = ((g.n[2] + BX - 1) / BX) * ((g.n[1] + BY - 1) / BY) * ((g.n[0] + BZ - 1) / BZ);
  // 16-byte copies need n2 % 4 == 0 (rows of whole chunks), no chunk across the periodic seam
  // (n2 >= TXA) and 16-byte aligned field pointers
  const bool aligned = ((reinterpret_cast<uintptr_t>(f) | reinterpret_cast<uintptr_t>(mu ? mu : f)) & 15u) == 0;
  const int vec = (g.n[2] % 4 == 0 && g.n[2] >= TXA && g.n[1] >= TY && g.n[0] >= TZ && aligned) ? 1 : 0;
  note_launches(1);
  k_sl_tile<MODE><<<nb, 256, sm, st>>>(f, mu, disp, out, g.n[0], g.n[1], g.n[2], ht, vec);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_departure_tile(const Grid& g, const float* v, float* xm, float* xp, float ht, int both,
                                  cudaStream_t st) {
  const size_t sm = sizeof(float) * TILEA * 3;
  static std::atomic<bool> attr{false};
  if (!attr.load()) {
    cudaError_t e = cudaFuncSetAttribute(k_departure_tile, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    attr.store(true);
  }
  const int nb = ((g.n[2] + BX - 1) / BX) * ((g.n[1] + BY - 1) / BY) * ((g.n[0] + BZ - 1) / BZ);
  const bool aligned = (reinterpret_cast<uintptr_t>(v) & 15u) == 0;
  const int vec = (g.n[2] % 4 == 0 && g.n[2] >= TXA && g.n[1] >= TY && g.n[0] >= TZ && aligned) ? 1 : 0;
  note_launches(1);
  k_departure_tile<<<nb, 256, sm, st>>>(v, xm, xp, g.n[0], g.n[1], g.n[2], ht, both, vec);
  return cudaGetLastError();
}

cudaError_t launch_sl_tile(const Grid& g, int adjoint, int continuity, const float* f, const float* disp,
                           const float* mu, float* out, float ht, cudaStream_t st) {
  if (!adjoint) {
    return continuity ? launch_mode<1>(g, f, mu, disp, out, ht, st) : launch_mode<0>(g, f, mu, disp, out, ht, st);
  }
  return continuity ? launch_mode<3>(g, f, mu, disp, out, ht, st) : launch_mode<2>(g, f, mu, disp, out, ht, st);
}

}  // namespace ga
