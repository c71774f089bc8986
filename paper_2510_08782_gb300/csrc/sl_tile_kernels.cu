// Tiled FP32 semi-Lagrangian step for 3D grids (Sec. 2.2; same arithmetic as sl_kernels.cu).
//
// A CTA owns a brick of 32 x 8 x 8 voxels (x contiguous). It stages the brick plus a halo of
// H + 1 cells below and H + 2 above (H = 2) of the transported field into shared memory with
// periodic wrap; for the two-field steps it also stages the product field f * mu, formed once per
// staged cell, so both interpolants are plain weighted sums sharing one stencil. Each thread owns a
// column of 8 voxels along z. When all 8 departure points of a column lie inside the halo and share
// the same integer x and y offsets (the common case for smooth velocities), the column walks the z
// planes once: each plane's 4 x 4 stencil is loaded from shared memory once and applied to every
// voxel of the column whose stencil contains that plane. Other columns interpolate voxel by voxel
// from shared memory, and departure points outside the halo read the field from global memory, so
// any displacement is handled exactly.
#include <cuda_runtime.h>

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
__device__ __forceinline__ void cp_async_wait_all_but_one() { asm volatile("cp.async.wait_group 1;\n" ::); }

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
  if (vec) {  // 16-byte chunks: n2 % 4 == 0 and n2 >= TXA, so a chunk never straddles the wrap
    for (int c = threadIdx.x; c < TY * TZ * (TXA / 4); c += blockDim.x) {
      const int cx = c % (TXA / 4), row = c / (TXA / 4);
      const int ty = row % TY, tz = row / TY;
      const int gy = wrap_any(gy0 + ty, n1), gz = wrap_any(gz0 + tz, n0);
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
// Persistent CTAs loop over bricks; the tile of the next brick is copied asynchronously into the
// second shared-memory buffer while the current brick is interpolated.
template <int MODE>
__global__ void __launch_bounds__(256, 1)
k_sl_tile(const float* __restrict__ f, const float* __restrict__ mu, const float* __restrict__ disp,
          float* __restrict__ out, int n0, int n1, int n2, float ht, int vec) {
  constexpr int NF = (MODE == 1 || MODE == 2) ? 2 : 1;  // staged fields: f (and mu)
  extern __shared__ __align__(16) float smem[];
  // layout: two staging buffers of NF tiles each, then (two-field steps) the interleaved tile
  float2* s2 = reinterpret_cast<float2*>(smem + 2 * NF * TILEA);
  const long long nv = (long long)n0 * n1 * n2;
  const int nbx = (n2 + BX - 1) / BX, nby = (n1 + BY - 1) / BY, nbz = (n0 + BZ - 1) / BZ;
  const int nbricks = nbx * nby * nbz;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int lx = lane, ly = warp;

  int b = blockIdx.x;
  if (b < nbricks) {
    const BrickIdx bi = brick_of(b, nbx, nby);
    stage_async(smem, f, bi, n0, n1, n2, vec != 0);
    if (NF == 2) stage_async(smem + TILEA, mu, bi, n0, n1, n2, vec != 0);
  }
  cp_async_commit();
  for (int it = 0; b < nbricks; ++it, b += gridDim.x) {
    float* cur = smem + (it & 1) * NF * TILEA;
    float* nxt = smem + ((it + 1) & 1) * NF * TILEA;
    const int bn = b + gridDim.x;
    if (bn < nbricks) {
      const BrickIdx bi = brick_of(bn, nbx, nby);
      stage_async(nxt, f, bi, n0, n1, n2, vec != 0);
      if (NF == 2) stage_async(nxt + TILEA, mu, bi, n0, n1, n2, vec != 0);
    }
    cp_async_commit();
    const BrickIdx bi = brick_of(b, nbx, nby);
    const int gx = bi.bx * BX + lx, gy = bi.by * BY + ly;
    const bool active = gx < n2 && gy < n1;
    // displacement loads are issued before waiting for the tile
    float dz[BZ], dy[BZ], dx[BZ];
    int nvalid = 0;
    if (active) {
#pragma unroll
      for (int v = 0; v < BZ; ++v) {
        const int gz = bi.bz * BZ + v;
        if (gz < n0) {
          const long long idx = ((long long)gz * n1 + gy) * n2 + gx;
          dz[v] = disp[idx];
          dy[v] = disp[nv + idx];
          dx[v] = disp[2 * nv + idx];
          nvalid = v + 1;
        } else {  // beyond the grid: copy the first voxel so the column test ignores it
          dz[v] = dz[0];
          dy[v] = dy[0];
          dx[v] = dx[0];
        }
      }
    }
    cp_async_wait_all_but_one();
    __syncthreads();
    if (NF == 2) {  // interleave (f, f * mu) once per staged cell for the two-field steps
      for (int e = threadIdx.x; e < TILEA; e += blockDim.x) {
        const float fv = cur[e];
        s2[e] = make_float2(fv, fv * cur[TILEA + e]);
      }
      __syncthreads();
    }
    if (active) {
      const float* sf = cur;
      const float* sm = cur + TILEA;
      // Column window: per axis the integer offsets of the 8 voxels must lie in {f, f + 1} with
      // f in [-H, 0]; then every stencil of the column lies in the 5-wide window [f - 1, f + 3] and
      // each voxel's 4 Lagrange weights sit in 5 slots (one slot zero). The plane/voxel schedule is
      // then fixed at compile time.
      float fxmin = floorf(dx[0]), fxmax = fxmin, fymin = floorf(dy[0]), fymax = fymin, fzmin = floorf(dz[0]),
            fzmax = fzmin;
#pragma unroll
      for (int v = 1; v < BZ; ++v) {
        const float fx = floorf(dx[v]), fy = floorf(dy[v]), fz = floorf(dz[v]);
        fxmin = fminf(fxmin, fx);
        fxmax = fmaxf(fxmax, fx);
        fymin = fminf(fymin, fy);
        fymax = fmaxf(fymax, fy);
        fzmin = fminf(fzmin, fz);
        fzmax = fmaxf(fzmax, fz);
      }
      const bool fast = fxmax - fxmin <= 1.f && fymax - fymin <= 1.f && fzmax - fzmin <= 1.f && fxmin >= -H &&
                        fxmin <= 0.f && fymin >= -H && fymin <= 0.f && fzmin >= -H && fzmin <= 0.f;
      if (fast) {
        const int ix0 = lx + XOFF - 1 + (int)fxmin;  // tile x of the window start
        const int iy0 = ly + H + (int)fymin;
        const int zbase = H + (int)fzmin;  // tile plane of voxel 0's window start
        float wx[BZ][5], wy[BZ][5], wz[BZ][5], P[BZ], S[BZ];
#pragma unroll
        for (int v = 0; v < BZ; ++v) {
          float w4[4];
          const float fx = floorf(dx[v]), fy = floorf(dy[v]), fz = floorf(dz[v]);
          lagrange4(dx[v] - fx, w4);
          const bool ox = fx > fxmin;
          wx[v][0] = ox ? 0.f : w4[0];
#pragma unroll
          for (int a = 1; a < 4; ++a) wx[v][a] = ox ? w4[a - 1] : w4[a];
          wx[v][4] = ox ? w4[3] : 0.f;
          lagrange4(dy[v] - fy, w4);
          const bool oy = fy > fymin;
          wy[v][0] = oy ? 0.f : w4[0];
#pragma unroll
          for (int a = 1; a < 4; ++a) wy[v][a] = oy ? w4[a - 1] : w4[a];
          wy[v][4] = oy ? w4[3] : 0.f;
          lagrange4(dz[v] - fz, w4);
          const bool oz = fz > fzmin;
          wz[v][0] = oz ? 0.f : w4[0];
#pragma unroll
          for (int a = 1; a < 4; ++a) wz[v][a] = oz ? w4[a - 1] : w4[a];
          wz[v][4] = oz ? w4[3] : 0.f;
          P[v] = 0.f;
          S[v] = 0.f;
        }
#pragma unroll
        for (int k = 0; k < BZ + 4; ++k) {
          const int off = ((zbase + k) * TY + iy0) * TXA + ix0;
          float q[5][5], qp[5][5];
#pragma unroll
          for (int bb = 0; bb < 5; ++bb)
#pragma unroll
            for (int a = 0; a < 5; ++a) {
              if (NF == 2) {
                const float2 t = s2[off + bb * TXA + a];
                q[bb][a] = t.x;
                qp[bb][a] = t.y;
              } else {
                q[bb][a] = sf[off + bb * TXA + a];
              }
            }
#pragma unroll
          for (int v = 0; v < BZ; ++v) {
            const int r = k - v;  // compile time: plane k is slot r of voxel v's window
            if (r >= 0 && r < 5) {
              float sy = 0.f, syp = 0.f;
#pragma unroll
              for (int bb = 0; bb < 5; ++bb) {
                sy += wy[v][bb] * (wx[v][0] * q[bb][0] + wx[v][1] * q[bb][1] + wx[v][2] * q[bb][2] +
                                   wx[v][3] * q[bb][3] + wx[v][4] * q[bb][4]);
                if (NF == 2)
                  syp += wy[v][bb] * (wx[v][0] * qp[bb][0] + wx[v][1] * qp[bb][1] + wx[v][2] * qp[bb][2] +
                                      wx[v][3] * qp[bb][3] + wx[v][4] * qp[bb][4]);
              }
              P[v] += wz[v][r] * sy;
              if (NF == 2) S[v] += wz[v][r] * syp;
            }
          }
        }
#pragma unroll
        for (int v = 0; v < BZ; ++v)
          if (v < nvalid)
            store_step<MODE>(out, mu, ((long long)(bi.bz * BZ + v) * n1 + gy) * n2 + gx, P[v], S[v], ht);
      } else {
#pragma unroll 1
        for (int v = 0; v < nvalid; ++v) {
          float P = 0.f, S = 0.f;
          const long long vidx = ((long long)(bi.bz * BZ + v) * n1 + gy) * n2 + gx;
          const float vz = disp[vidx], vy = disp[nv + vidx], vx = disp[2 * nv + vidx];
          const float fz = floorf(vz), fy = floorf(vy), fx = floorf(vx);
          const bool inhalo = fz >= -H && fz <= H - 1 && fy >= -H && fy <= H - 1 && fx >= -H && fx <= H - 1;
          if (inhalo) {
            float wz[4], wy[4], wx[4];
            lagrange4(vz - fz, wz);
            lagrange4(vy - fy, wy);
            lagrange4(vx - fx, wx);
            const int iz0 = v + H + (int)fz, iy0 = ly + H + (int)fy, ix0 = lx + XOFF - 1 + (int)fx;
            for (int c = 0; c < 4; ++c) {
              float ay = 0.f, ayp = 0.f;
              for (int bb = 0; bb < 4; ++bb) {
                const int o = ((iz0 + c) * TY + iy0 + bb) * TXA + ix0;
                float sx = 0.f, sxp = 0.f;
                for (int a = 0; a < 4; ++a) {
                  sx += wx[a] * sf[o + a];
                  if (NF == 2) sxp += wx[a] * sf[o + a] * sm[o + a];
                }
                ay += wy[bb] * sx;
                if (NF == 2) ayp += wy[bb] * sxp;
              }
              P += wz[c] * ay;
              if (NF == 2) S += wz[c] * ayp;
            }
          } else {
            gather_global<NF>(f, mu, bi.bz * BZ + v, gy, gx, vz, vy, vx, n0, n1, n2, P, S);
          }
          store_step<MODE>(out, mu, vidx, P, S, ht);
        }
      }
    }
    __syncthreads();  // the buffer just read is refilled by the next iteration's prefetch
  }
  asm volatile("cp.async.wait_all;\n" ::);
}

template <int MODE>
cudaError_t launch_mode(const Grid& g, const float* f, const float* mu, const float* disp, float* out, float ht,
                        cudaStream_t st) {
  constexpr int NF = (MODE == 1 || MODE == 2) ? 2 : 1;
  const size_t sm = sizeof(float) * TILEA * NF * 2 + (NF == 2 ? sizeof(float2) * TILEA : 0);
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_sl_tile<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const int nb = ((g.n[2] + BX - 1) / BX) * ((g.n[1] + BY - 1) / BY) * ((g.n[0] + BZ - 1) / BZ);
  const int grid = nb < 152 ? nb : 152;
  // 16-byte copies need n2 % 4 == 0 (rows of whole chunks), no chunk across the periodic seam
  // (n2 >= TXA) and 16-byte aligned field pointers
  const bool aligned = ((reinterpret_cast<uintptr_t>(f) | reinterpret_cast<uintptr_t>(mu ? mu : f)) & 15u) == 0;
  const int vec = (g.n[2] % 4 == 0 && g.n[2] >= TXA && aligned) ? 1 : 0;
  note_launches(1);
  k_sl_tile<MODE><<<grid, 256, sm, st>>>(f, mu, disp, out, g.n[0], g.n[1], g.n[2], ht, vec);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_sl_tile(const Grid& g, int adjoint, int continuity, const float* f, const float* disp,
                           const float* mu, float* out, float ht, cudaStream_t st) {
  if (!adjoint) {
    return continuity ? launch_mode<1>(g, f, mu, disp, out, ht, st) : launch_mode<0>(g, f, mu, disp, out, ht, st);
  }
  return continuity ? launch_mode<3>(g, f, mu, disp, out, ht, st) : launch_mode<2>(g, f, mu, disp, out, ht, st);
}

}  // namespace ga
