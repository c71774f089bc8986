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
constexpr int kTileThreads = 32 * BY;  // one warp per brick row
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

// Output of one step from P = I[f], S = I[f mu] at the departure point and m = mu at the voxel.
template <int MODE> __device__ __forceinline__ float step_value(float P, float S, float m, float ht) {
  if (MODE == 1) return P - 0.5f * ht * (S + m * (P - ht * S));
  if (MODE == 2) return P + 0.5f * ht * (S + m * (P + ht * S));
  return P;
}

template <int MODE>
__device__ __forceinline__ void store_step(float* __restrict__ out, const float* __restrict__ mu, long long idx,
                                           float P, float S, float ht, float2* __restrict__ qout) {
  const float m = (MODE == 1 || MODE == 2) ? mu[idx] : 0.f;
  const float y = step_value<MODE>(P, S, m, ht);
  out[idx] = y;
  if ((MODE == 1 || MODE == 2) && qout) qout[idx] = make_float2(y, y * m);
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
// Two-field steps interleave (f, f mu) into 8-byte pairs with their own row pitch TXP (>= TXA). A
// half-warp's 64-bit loads cover 16 consecutive pairs; with the row and plane pitches multiples of 16
// pairs (TXP = 48), lanes whose stencils start on different rows or planes fall on different banks.
// Measured at 256^3: 48 -> 0.334 ms, 40 -> 0.345 ms, 41 -> 0.361 ms, 44 -> 0.364 ms. 3 CTAs of
// 75 KB still fit on an SM.
constexpr int TXP = 48;

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

// Tile planes and elements of a brick of depth ZB (z voxels per thread).
template <int ZB> struct Tile {
  static constexpr int TZ = ZB + 2 * H + 2;
  static constexpr int A = TXA * TY * TZ;  // floats of one staged field
  static constexpr int P = TXP * TY * TZ;  // (f, f mu) pairs of the two-field steps
};

// Issue the copies of one brick's tile of `src` into `dst` (all threads of the CTA).
template <int ZB = BZ>
__device__ __forceinline__ void stage_async(float* dst, const float* __restrict__ src, const BrickIdx& bi, int n0,
                                            int n1, int n2, bool vec) {
  constexpr int TZ = Tile<ZB>::TZ, TILEA = Tile<ZB>::A;
  const int gx0 = bi.bx * BX - XOFF, gy0 = bi.by * BY - H - 1, gz0 = bi.bz * ZB - H - 1;
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
      cp_async16(dst + row * TXA + 4 * cx, src + ((gz * n1 + gy) * n2 + gx));  // < 2^30: axes <= 1024
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

// Issue the copies of one brick's tile of (f, f mu) pairs from `src` into the pair layout (row pitch TXP)
// at `dst` (all threads of the CTA): the two-field steps' tile without the interleaving pass.
__device__ __forceinline__ void cp_async8(float2* sdst, const float2* gsrc) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gsrc));
}
template <int ZB>
__device__ __forceinline__ void stage_pairs_async(float2* dst, const float2* __restrict__ src, const BrickIdx& bi,
                                                  int n0, int n1, int n2, bool vec) {
  constexpr int TZ = Tile<ZB>::TZ;
  const int gx0 = bi.bx * BX - XOFF, gy0 = bi.by * BY - H - 1, gz0 = bi.bz * ZB - H - 1;
  if (vec) {  // 16-byte chunks of two pairs: n2 % 4 == 0 and n2 >= TXA (see stage_async)
    for (int c = threadIdx.x; c < TY * TZ * (TXA / 2); c += blockDim.x) {
      const int cx = c % (TXA / 2), row = c / (TXA / 2);
      const int ty = row % TY, tz = row / TY;
      int gy = gy0 + ty, gz = gz0 + tz;
      gy = gy < 0 ? gy + n1 : (gy >= n1 ? gy - n1 : gy);
      gz = gz < 0 ? gz + n0 : (gz >= n0 ? gz - n0 : gz);
      int gx = gx0 + 2 * cx;
      gx = gx < 0 ? gx + n2 : (gx >= n2 ? gx - n2 : gx);
      cp_async16(reinterpret_cast<float*>(dst + row * TXP + 2 * cx),
                 reinterpret_cast<const float*>(src + ((gz * n1 + gy) * n2 + gx)));  // < 2^30: axes <= 1024
    }
  } else {
    for (int e = threadIdx.x; e < TXA * TY * TZ; e += blockDim.x) {
      const int tx = e % TXA, row = e / TXA;
      const int ty = row % TY, tz = row / TY;
      const int gy = wrap_any(gy0 + ty, n1), gz = wrap_any(gz0 + tz, n0);
      const int gx = wrap_any(gx0 + tx, n2);
      cp_async8(dst + row * TXP + tx, src + ((size_t)gz * n1 + gy) * n2 + gx);
    }
  }
}

// ---- scalar / packed-pair arithmetic with explicit rounding ----
// The pair type float2 runs two independent lanes through the FP32x2 FMA path of sm_100+; the scalar
// overloads perform the same operations in the same order, so a voxel's interpolant does not depend
// on whether it was computed alone or in a pair.
__device__ __forceinline__ float vfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float vmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float2 vmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float vadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float2 vadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
template <typename V> __device__ __forceinline__ V vsplat(float c);
template <> __device__ __forceinline__ float vsplat<float>(float c) { return c; }
template <> __device__ __forceinline__ float2 vsplat<float2>(float c) { return make_float2(c, c); }

// Cubic Lagrange weights on the nodes -1, 0, 1, 2 at offset t in [0, 1):
// w_-1 = -t(t-1)(t-2)/6, w_0 = (t+1)(t-1)(t-2)/2, w_1 = -(t+1)t(t-2)/2, w_2 = (t+1)t(t-1)/6.
template <typename V> __device__ __forceinline__ void lagrange4v(V t, V* w) {
  const V tp1 = vadd(t, vsplat<V>(1.f)), tm1 = vadd(t, vsplat<V>(-1.f)), tm2 = vadd(t, vsplat<V>(-2.f));
  const V a = vmul(t, tm1), b = vmul(tp1, tm2);
  w[0] = vmul(vmul(a, tm2), vsplat<V>(-1.f / 6.f));
  w[1] = vmul(vmul(b, tm1), vsplat<V>(0.5f));
  w[2] = vmul(vmul(b, t), vsplat<V>(-0.5f));
  w[3] = vmul(vmul(a, tp1), vsplat<V>(1.f / 6.f));
}

// Tensor-product sum of the 4 x 4 x 4 taps returned by ld(offset) (offset relative to the stencil's
// first tap, in tile elements; PITCH elements per tile row): 16 rows along x, then 4 columns along y,
// then z.
template <int PITCH, typename V, typename Load>
__device__ __forceinline__ V interp64(const V* wz, const V* wy, const V* wx, Load ld) {
  V acc;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    V ay;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int o = (c * TY + b) * PITCH;
      V r = vmul(ld(o), wx[0]);
      r = vfma(ld(o + 1), wx[1], r);
      r = vfma(ld(o + 2), wx[2], r);
      r = vfma(ld(o + 3), wx[3], r);
      ay = b == 0 ? vmul(r, wy[0]) : vfma(r, wy[b], ay);
    }
    acc = c == 0 ? vmul(ay, wz[0]) : vfma(ay, wz[c], acc);
  }
  return acc;
}

__device__ __forceinline__ bool in_halo(float fz, float fy, float fx) {
  return fz >= -H && fz <= H - 1 && fy >= -H && fy <= H - 1 && fx >= -H && fx <= H - 1;
}

// One voxel (brick-local z index v, global index idx): shared-memory taps when the stencil lies in the
// halo, global taps otherwise. Two-field steps read the interleaved (f, f mu) tile `sf`.
template <int MODE>
__device__ __forceinline__ void sl_single(const float* __restrict__ f, const float* __restrict__ mu,
                                          float* __restrict__ out, float2* __restrict__ qout, const float* sf, int col,
                                          long long idx, int gz, int v, int gy, int gx, float vz, float vy, float vx,
                                          int n0, int n1, int n2, float ht) {
  constexpr int NF = (MODE == 1 || MODE == 2) ? 2 : 1;
  const float fz = floorf(vz), fy = floorf(vy), fx = floorf(vx);
  float P = 0.f, S = 0.f;
  if (in_halo(fz, fy, fx)) {
    float wz[4], wy[4], wx[4];
    lagrange4v(vz - fz, wz);
    lagrange4v(vy - fy, wy);
    lagrange4v(vx - fx, wx);
    if (NF == 2) {  // col is the pair-layout index here
      const int base = col + ((v + H + (int)fz) * TY + (int)fy) * TXP + (int)fx;
      P = interp64<TXP, float>(wz, wy, wx, [&](int o) { return sf[2 * (base + o)]; });
      S = interp64<TXP, float>(wz, wy, wx, [&](int o) { return sf[2 * (base + o) + 1]; });
    } else {
      const int base = col + ((v + H + (int)fz) * TY + (int)fy) * TXA + (int)fx;
      P = interp64<TXA, float>(wz, wy, wx, [&](int o) { return sf[base + o]; });
    }
  } else {
    gather_global<NF>(f, mu, gz, gy, gx, vz, vy, vx, n0, n1, n2, P, S);
  }
  store_step<MODE>(out, mu, idx, P, S, ht, qout);
}

// MODE 0: advection state step          out = I[f](X-)
// MODE 1: continuity state step         out = P - ht/2 (S + mu (P - ht S)),  P = I[f], S = I[f mu]
// MODE 2: advection adjoint step        out = L + ht/2 (S + mu (L + ht S)),  L = I[f], S = I[f mu]
// MODE 3: continuity adjoint step       out = I[f](X+)
// One CTA per brick. The tile (and, for the two-field steps, mu) is copied asynchronously into
// shared memory; several CTAs per SM overlap one brick's copies with another's interpolation. For
// the two-field steps the staged mu tile is then overwritten with f * mu, so the product is formed
// once per tile element. Each thread walks its column of 8 voxels two at a time: the pair's weights
// and its 64-tap sums (per field) run as packed FP32x2 operations, with the taps read from shared
// memory at compile-time offsets from one base index per voxel.
template <int MODE, int ZB>
__device__ __forceinline__ void sl_tile_body(const float* __restrict__ f, const float* __restrict__ mu,
                                             const float* __restrict__ disp, float* __restrict__ out, int n0, int n1,
                                             int n2, float ht, int vec, const float2* __restrict__ qin,
                                             float2* __restrict__ qout) {
  constexpr int NF = (MODE == 1 || MODE == 2) ? 2 : 1;  // staged fields: f (and f * mu)
  constexpr int TILEA = Tile<ZB>::A;
  extern __shared__ __align__(16) float smem[];
  const float* sf = smem;
  const float2* sp = reinterpret_cast<const float2*>(smem);  // two-field steps: (f, f mu) per element
  const long long nv = (long long)n0 * n1 * n2;
  const long long plane = (long long)n1 * n2;
  const int nbx = (n2 + BX - 1) / BX, nby = (n1 + BY - 1) / BY;
  const BrickIdx bi = brick_of(blockIdx.x, nbx, nby);
  const bool pairs_in = NF == 2 && qin != nullptr;  // the previous step wrote (f, f mu): stage them as they are
  if (pairs_in) {
    stage_pairs_async<ZB>(reinterpret_cast<float2*>(smem), qin, bi, n0, n1, n2, vec != 0);
  } else {
    stage_async<ZB>(smem, f, bi, n0, n1, n2, vec != 0);
    if (NF == 2) stage_async<ZB>(smem + TILEA, mu, bi, n0, n1, n2, vec != 0);
  }
  cp_async_commit();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int gx = bi.bx * BX + lane, gy = bi.by * BY + warp;
  const bool active = gx < n2 && gy < n1;
  const int nz = min(ZB, n0 - bi.bz * ZB);
  const long long idx0 = ((long long)(bi.bz * ZB) * n1 + gy) * n2 + gx;
  // This column's fields from per-thread base pointers with 32-bit offsets v * pl (an axis has at most
  // 1024 points, so a field's offsets fit in 32 bits).
  const int pl = n1 * n2;
  const float* dz0 = disp + idx0;
  const float* dy0 = dz0 + nv;
  const float* dx0 = dy0 + nv;
  const float* mu0 = NF == 2 ? mu + idx0 : nullptr;
  float* out0 = out + idx0;
  float2* q0 = (NF == 2 && qout) ? qout + idx0 : nullptr;
  // Displacements (and mu at the voxel) of one pair ahead are kept in registers: the first pair's are
  // requested while the tile is still being copied, each later pair's while the previous one is
  // interpolated.
  float za = 0.f, zb = 0.f, ya = 0.f, yb = 0.f, xa = 0.f, xb = 0.f, ma = 0.f, mb = 0.f;
  auto fetch = [&](int v) {
    const int oa = v * pl, ob = oa + pl;
    za = dz0[oa], zb = dz0[ob];
    ya = dy0[oa], yb = dy0[ob];
    xa = dx0[oa], xb = dx0[ob];
    if (NF == 2) ma = mu0[oa], mb = mu0[ob];
  };
  if (NF == 1 && active && nz >= 2) fetch(0);
  if (NF == 2 && active && nz >= 2) {
    // the first pair's loads follow the tile conversion (which needs the registers): pull their lines
    // into L2 now, while the tile copies are in flight
#pragma unroll
    for (int c = 0; c < 4; ++c) {  // the three displacement components, then mu
      const float* base = c < 3 ? disp + c * nv + idx0 : mu + idx0;
      asm volatile("prefetch.global.L2 [%0];\n" ::"l"(base));
      asm volatile("prefetch.global.L2 [%0];\n" ::"l"(base + plane));
    }
  }
  asm volatile("cp.async.wait_all;\n" ::);
  __syncthreads();
  if (pairs_in) {
    if (active && nz >= 2) fetch(0);
  } else if (NF == 2) {
    // Interleave in place: the f and mu tiles (TILEA floats each) become TILEA pairs (f, f mu) over the
    // same bytes, so a tap of both fields is one 64-bit shared load. Every thread holds its elements
    // in registers across the barrier, since a pair overwrites other threads' source elements.
    constexpr int PER = (TILEA + kTileThreads - 1) / kTileThreads;
    float fa[PER], fm[PER];
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      const int e = threadIdx.x + kTileThreads * i;
      if (e < TILEA) {
        fa[i] = smem[e];
        fm[i] = fa[i] * smem[TILEA + e];
      }
    }
    __syncthreads();
    float2* pw = reinterpret_cast<float2*>(smem);
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      const int e = threadIdx.x + kTileThreads * i;
      if (e < TILEA) pw[TXP == TXA ? e : (e / TXA) * TXP + e % TXA] = make_float2(fa[i], fm[i]);
    }
    if (active && nz >= 2) fetch(0);  // after the conversion, whose registers it would otherwise share
    __syncthreads();
  }
  if (!active) return;
  // tile index of (z = 0, y, x) minus the x tap offset (in the pair layout for two-field steps)
  const int col = (warp + H) * (NF == 2 ? TXP : TXA) + lane + XOFF - 1;

  int v = 0;
#pragma unroll 1
  for (; v + 1 < nz; v += 2) {
    const int oa = v * pl, ob = oa + pl;
    const float cza = za, czb = zb, cya = ya, cyb = yb, cxa = xa, cxb = xb, cma = ma, cmb = mb;
    if (v + 3 < nz) fetch(v + 2);
    const float fza = floorf(cza), fya = floorf(cya), fxa = floorf(cxa);
    const float fzb = floorf(czb), fyb = floorf(cyb), fxb = floorf(cxb);
    if (in_halo(fza, fya, fxa) && in_halo(fzb, fyb, fxb)) {
      constexpr int PT = NF == 2 ? TXP : TXA;
      const int ba = col + ((v + H + (int)fza) * TY + (int)fya) * PT + (int)fxa;
      const int bb = col + ((v + 1 + H + (int)fzb) * TY + (int)fyb) * PT + (int)fxb;
      float2 wz[4], wy[4], wx[4];
      if (NF == 2) {
        // per voxel, the two fields as one packed pair; the weights carry the voxel's value in both
        // lanes (computed as a pair of equal arguments), so each lane repeats the scalar arithmetic
        lagrange4v(vsplat<float2>(cza - fza), wz);
        lagrange4v(vsplat<float2>(cya - fya), wy);
        lagrange4v(vsplat<float2>(cxa - fxa), wx);
        const float2 A = interp64<TXP, float2>(wz, wy, wx, [&](int o) { return sp[ba + o]; });
        const float ya = step_value<MODE>(A.x, A.y, cma, ht);
        out0[oa] = ya;
        if (q0) q0[oa] = make_float2(ya, ya * cma);
        lagrange4v(vsplat<float2>(czb - fzb), wz);
        lagrange4v(vsplat<float2>(cyb - fyb), wy);
        lagrange4v(vsplat<float2>(cxb - fxb), wx);
        const float2 B = interp64<TXP, float2>(wz, wy, wx, [&](int o) { return sp[bb + o]; });
        const float yb = step_value<MODE>(B.x, B.y, cmb, ht);
        out0[ob] = yb;
        if (q0) q0[ob] = make_float2(yb, yb * cmb);
      } else {  // one field: the pair of voxels as one packed pair
        lagrange4v(make_float2(cza - fza, czb - fzb), wz);
        lagrange4v(make_float2(cya - fya, cyb - fyb), wy);
        lagrange4v(make_float2(cxa - fxa, cxb - fxb), wx);
        const float2 P = interp64<TXA, float2>(wz, wy, wx, [&](int o) { return make_float2(sf[ba + o], sf[bb + o]); });
        out0[oa] = step_value<MODE>(P.x, 0.f, cma, ht);
        out0[ob] = step_value<MODE>(P.y, 0.f, cmb, ht);
      }
    } else {
      const long long ia = idx0 + oa, ib = idx0 + ob;
      sl_single<MODE>(f, mu, out, qout, sf, col, ia, bi.bz * ZB + v, v, gy, gx, cza, cya, cxa, n0, n1, n2, ht);
      sl_single<MODE>(f, mu, out, qout, sf, col, ib, bi.bz * ZB + v + 1, v + 1, gy, gx, czb, cyb, cxb, n0, n1, n2, ht);
    }
  }
  if (v < nz) {
    const long long ia = idx0 + v * plane;
    sl_single<MODE>(f, mu, out, qout, sf, col, ia, bi.bz * ZB + v, v, gy, gx, disp[ia], disp[nv + ia], disp[2 * nv + ia],
                    n0, n1, n2, ht);
  }
}

// ---- column-reuse gather ------------------------------------------------------------------------
// With departure points less than a cell or so from the arrival points, the stencil base offsets
// (floors) of a thread's column of BZ voxels take at most two neighbouring values per axis. Each
// voxel's 4 x 4 x 4 stencil then lies in the column's padded 5 x 5 x 5 window: the base B is the
// smaller floor and a voxel whose floor is B + 1 takes its cubic weights shifted by one, with a zero
// in front (others end in a zero). The thread walks the BZ + 4 planes of the column once, reads each
// plane's 5 x 5 patch of (y, x) taps from shared memory once, and accumulates it into every voxel
// whose padded z-window holds that plane: 25 x (BZ + 4) / BZ = 37.5 taps per voxel instead of 64.
// The extra terms are exact zeros (w * t with w = 0 adds nothing), and the remaining products and
// sums run in the order of the per-voxel gather (x, then y, then z, first term a product), so every
// value equals the per-voxel gather's bit for bit. The walk trades shared-memory reads for FMAs
// (125 instead of 64 per field and voxel): it pays in the departure-point kernel, whose three velocity
// interpolants per sign share one stencil, and not in the one- and two-field transport steps, which
// keep the per-voxel gather.

// Column bases of one axis: B = min(floor) (or 0 when every floor is 1), valid when every floor is
// B or B + 1 and the padded window [B - 1, B + 3] stays inside the staged halo.
__device__ __forceinline__ bool column_base(float lo, float hi, int& B) {
  B = (int)fminf(lo, 0.f);
  return lo >= -(float)H && hi <= (float)(H - 1) && hi - lo <= 1.f;
}

// Padded weights of one axis: the cubic weights at t, placed at [sel, sel + 4) of five.
__device__ __forceinline__ void padded5(float t, bool sel, float* w5) {
  float w[4];
  lagrange4v(t, w);
  w5[0] = sel ? 0.f : w[0];
  w5[1] = sel ? w[0] : w[1];
  w5[2] = sel ? w[1] : w[2];
  w5[3] = sel ? w[2] : w[3];
  w5[4] = sel ? w[3] : 0.f;
}

// The whole column of BZ voxels of one thread by the padded-window walk, for NF fields that share the
// interpolation weights: disp(v, d) gives voxel v's displacement (z, y, x; cells), tap(i, t) reads the
// NF fields' values at tile index i (tile pitch PT) into t[0..NF), and emit(v, acc) receives voxel v's
// NF interpolants once its five planes are summed. Returns false, having done nothing, unless every
// active lane of the warp qualifies (the caller then gathers voxel by voxel).
template <int NF, int PT, typename Disp, typename Tap, typename Emit>
__device__ __forceinline__ bool column_walk(int col, Disp&& disp, Tap&& tap, Emit&& emit) {
  float lz = 1e30f, hz = -1e30f, ly = 1e30f, hy = -1e30f, lx = 1e30f, hx = -1e30f;
#pragma unroll
  for (int v = 0; v < BZ; ++v) {
    float d[3];
    disp(v, d);
    const float a = floorf(d[0]), b = floorf(d[1]), c = floorf(d[2]);
    lz = fminf(lz, a), hz = fmaxf(hz, a);
    ly = fminf(ly, b), hy = fmaxf(hy, b);
    lx = fminf(lx, c), hx = fmaxf(hx, c);
  }
  int Bz, By, Bx;
  bool ok = column_base(lz, hz, Bz);
  ok = column_base(ly, hy, By) && ok;
  ok = column_base(lx, hx, Bx) && ok;
  // NaN displacements fail every comparison above, so such a column takes the per-voxel path
  if (!__all_sync(__activemask(), ok)) return false;
  // tile index of the first padded tap of voxel 0
  const int base = col + ((H + Bz) * TY + By) * PT + Bx;
  float wx[BZ][5], wy[BZ][5], wz[BZ][5];
  float acc[BZ][NF];
#pragma unroll
  for (int P = 0; P < BZ + 4; ++P) {
    if (P < BZ) {  // voxel P enters: its padded weights
      float d[3];
      disp(P, d);
      const float fz = floorf(d[0]), fy = floorf(d[1]), fx = floorf(d[2]);
      padded5(d[0] - fz, fz > (float)Bz, wz[P]);
      padded5(d[1] - fy, fy > (float)By, wy[P]);
      padded5(d[2] - fx, fx > (float)Bx, wx[P]);
    }
    float ys[BZ][NF];
#pragma unroll
    for (int b = 0; b < 5; ++b) {
      float t[5][NF];
      const int o = base + (P * TY + b) * PT;
#pragma unroll
      for (int a = 0; a < 5; ++a) tap(o + a, t[a]);
#pragma unroll
      for (int v = 0; v < BZ; ++v) {
        if (v > P || v < P - 4) continue;
#pragma unroll
        for (int f = 0; f < NF; ++f) {
          float r = __fmul_rn(t[0][f], wx[v][0]);
          r = __fmaf_rn(t[1][f], wx[v][1], r);
          r = __fmaf_rn(t[2][f], wx[v][2], r);
          r = __fmaf_rn(t[3][f], wx[v][3], r);
          r = __fmaf_rn(t[4][f], wx[v][4], r);
          ys[v][f] = b == 0 ? __fmul_rn(r, wy[v][0]) : __fmaf_rn(r, wy[v][b], ys[v][f]);
        }
      }
    }
#pragma unroll
    for (int v = 0; v < BZ; ++v) {
      if (v > P || v < P - 4) continue;
#pragma unroll
      for (int f = 0; f < NF; ++f)
        acc[v][f] = P == v ? __fmul_rn(ys[v][f], wz[v][0]) : __fmaf_rn(ys[v][f], wz[v][P - v], acc[v][f]);
    }
    if (P >= 4) emit(P - 4, acc[P - 4]);  // voxel P - 4 has seen its five planes
  }
  return true;
}

// Two-field steps (MODE 1, 2) fit 3 CTAs per SM by shared memory; one-field steps (MODE 0, 3) fit 4
// when held to 64 registers.
template <int MODE, int ZB>
__global__ void __launch_bounds__(256, ZB <= 8 ? 3 : 2) k_sl_tile2(const float* __restrict__ f,
                                                                  const float* __restrict__ mu,
                                                                  const float* __restrict__ disp,
                                                                  float* __restrict__ out, int n0, int n1, int n2,
                                                                  float ht, int vec, const float2* __restrict__ qin,
                                                                  float2* __restrict__ qout) {
  sl_tile_body<MODE, ZB>(f, mu, disp, out, n0, n1, n2, ht, vec, qin, qout);
}
template <int MODE, int ZB>
__global__ void __launch_bounds__(256, 4) k_sl_tile1(const float* __restrict__ f, const float* __restrict__ mu,
                                                     const float* __restrict__ disp, float* __restrict__ out, int n0,
                                                     int n1, int n2, float ht, int vec, const float2* __restrict__ qin,
                                                     float2* __restrict__ qout) {
  sl_tile_body<MODE, ZB>(f, mu, disp, out, n0, n1, n2, ht, vec, qin, qout);
}

// RK2 departure points (displacements in cells) for 3D FP32 grids: X* = x -/+ h_t v(x), then
// X-/+ = x -/+ (h_t / 2)(v(x) + I[v](X*)). The three velocity components of the brick + halo are
// staged in shared memory; the three interpolants at X* share one stencil. A full column whose warp
// qualifies takes the padded-window walk (column_walk) for each sign; otherwise each thread walks its
// column two voxels at a time: a pair's weights and its 64-tap sums run as packed FP32x2 operations
// (interp64, as in the state steps). A voxel done alone (odd column length, or a stencil beyond the
// halo in the pair) repeats the same operations in scalar form, so its value does not depend on the
// pairing.
__global__ void __launch_bounds__(256, 2)
k_departure_tile(const float* __restrict__ v, float* __restrict__ xm, float* __restrict__ xp, int n0, int n1, int n2,
                 float ht, int both, int vec) {
  extern __shared__ __align__(16) float smem[];
  const long long nv = (long long)n0 * n1 * n2;
  const long long plane = (long long)n1 * n2;
  const int nbx = (n2 + BX - 1) / BX, nby = (n1 + BY - 1) / BY;
  const BrickIdx bi = brick_of(blockIdx.x, nbx, nby);
  for (int c = 0; c < 3; ++c) stage_async<BZ>(smem + c * TILEA, v + c * nv, bi, n0, n1, n2, vec != 0);
  cp_async_commit();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int gx = bi.bx * BX + lane, gy = bi.by * BY + warp;
  const float twopi = 6.283185307179586f;
  const float ih[3] = {(float)n0 / twopi, (float)n1 / twopi, (float)n2 / twopi};  // 1 / h_a
  asm volatile("cp.async.wait_all;\n" ::);
  __syncthreads();
  if (gx >= n2 || gy >= n1) return;
  const int nz = min(BZ, n0 - bi.bz * BZ);
  const long long idx0 = ((long long)(bi.bz * BZ) * n1 + gy) * n2 + gx;
  // tile index of (z = 0, y, x) minus the stencil's first-tap offset
  const int col = (warp + H) * TXA + lane + XOFF - 1;
  auto center = [&](int vz, int k) { return smem[k * TILEA + ((vz + H + 1) * TY + warp + H + 1) * TXA + lane + XOFF]; };
  // one voxel alone
  auto single = [&](int vz, float sign, float* o) {
    const long long idx = idx0 + vz * plane;
    float d[3], vc[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      vc[k] = center(vz, k);
      d[k] = -sign * ht * vc[k] * ih[k];
    }
    const float fz = floorf(d[0]), fy = floorf(d[1]), fx = floorf(d[2]);
    if (in_halo(fz, fy, fx)) {
      float wz[4], wy[4], wx[4];
      lagrange4v(d[0] - fz, wz);
      lagrange4v(d[1] - fy, wy);
      lagrange4v(d[2] - fx, wx);
      const int base = col + ((vz + H + (int)fz) * TY + (int)fy) * TXA + (int)fx;
#pragma unroll 1
      for (int k = 0; k < 3; ++k) {
        const float* t = smem + k * TILEA + base;
        const float acc = interp64<TXA, float>(wz, wy, wx, [&](int q) { return t[q]; });
        o[k * nv + idx] = -sign * 0.5f * ht * (vc[k] + acc) * ih[k];
      }
    } else {
#pragma unroll 1
      for (int k = 0; k < 3; ++k) {
        float P, S;
        gather_global<1>(v + k * nv, nullptr, bi.bz * BZ + vz, gy, gx, d[0], d[1], d[2], n0, n1, n2, P, S);
        o[k * nv + idx] = -sign * 0.5f * ht * (vc[k] + P) * ih[k];
      }
    }
  };
#pragma unroll 1
  for (int sg = 0; sg < (both ? 2 : 1); ++sg) {
    const float sign = sg == 0 ? 1.f : -1.f;
    float* o = sg == 0 ? xm : xp;
    if (nz == BZ) {  // the column walk over the three velocity tiles (X* within a cell or so)
      auto disp = [&](int vz, float* d) {
#pragma unroll
        for (int k = 0; k < 3; ++k) d[k] = -sign * ht * center(vz, k) * ih[k];
      };
      auto tap = [&](int i, float* t) {
#pragma unroll
        for (int k = 0; k < 3; ++k) t[k] = smem[k * TILEA + i];
      };
      auto emit = [&](int vz, const float* acc) {
        const long long idx = idx0 + vz * plane;
#pragma unroll
        for (int k = 0; k < 3; ++k) o[k * nv + idx] = -sign * 0.5f * ht * (center(vz, k) + acc[k]) * ih[k];
      };
      if (column_walk<3, TXA>(col, disp, tap, emit)) continue;
    }
    int vz = 0;
#pragma unroll 1
    for (; vz + 1 < nz; vz += 2) {
      float da[3], db[3], ca[3], cb[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        ca[k] = center(vz, k);
        cb[k] = center(vz + 1, k);
        da[k] = -sign * ht * ca[k] * ih[k];
        db[k] = -sign * ht * cb[k] * ih[k];
      }
      const float fza = floorf(da[0]), fya = floorf(da[1]), fxa = floorf(da[2]);
      const float fzb = floorf(db[0]), fyb = floorf(db[1]), fxb = floorf(db[2]);
      if (in_halo(fza, fya, fxa) && in_halo(fzb, fyb, fxb)) {
        float2 wz[4], wy[4], wx[4];
        lagrange4v(make_float2(da[0] - fza, db[0] - fzb), wz);
        lagrange4v(make_float2(da[1] - fya, db[1] - fyb), wy);
        lagrange4v(make_float2(da[2] - fxa, db[2] - fxb), wx);
        const int ba = col + ((vz + H + (int)fza) * TY + (int)fya) * TXA + (int)fxa;
        const int bb = col + ((vz + 1 + H + (int)fzb) * TY + (int)fyb) * TXA + (int)fxb;
        const long long ia = idx0 + vz * plane, ib = ia + plane;
#pragma unroll 1
        for (int k = 0; k < 3; ++k) {
          const float* t = smem + k * TILEA;
          const float2 acc =
              interp64<TXA, float2>(wz, wy, wx, [&](int q) { return make_float2(t[ba + q], t[bb + q]); });
          o[k * nv + ia] = -sign * 0.5f * ht * (ca[k] + acc.x) * ih[k];
          o[k * nv + ib] = -sign * 0.5f * ht * (cb[k] + acc.y) * ih[k];
        }
      } else {
        single(vz, sign, o);
        single(vz + 1, sign, o);
      }
    }
    if (vz < nz) single(vz, sign, o);
  }
}

template <int MODE, int ZB>
cudaError_t launch_mode_zb(const Grid& g, const float* f, const float* mu, const float* disp, float* out, float ht,
                           const float2* qin, float2* qout, cudaStream_t st) {
  constexpr int NF = (MODE == 1 || MODE == 2) ? 2 : 1;
  constexpr int TILEA = Tile<ZB>::A, TILEP = Tile<ZB>::P;
  // two-field steps: the f and mu tiles, then the same bytes (plus row padding) as (f, f mu) pairs
  const size_t sm = NF == 2 ? sizeof(float) * (2 * TILEP > 2 * TILEA ? 2 * TILEP : 2 * TILEA) : sizeof(float) * TILEA;
  void (*kern)(const float*, const float*, const float*, float*, int, int, int, float, int, const float2*, float2*);
  if constexpr (NF == 2) kern = k_sl_tile2<MODE, ZB>;
  else kern = k_sl_tile1<MODE, ZB>;
  static std::atomic<bool> attr{false};
  if (!attr.load()) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    attr.store(true);
  }
  const int nb = ((g.n[2] + BX - 1) / BX) * ((g.n[1] + BY - 1) / BY) * ((g.n[0] + ZB - 1) / ZB);
  // 16-byte copies need n2 % 4 == 0 (rows of whole chunks), no chunk across the periodic seam
  // (n2 >= TXA) and 16-byte aligned field pointers
  const bool aligned = ((reinterpret_cast<uintptr_t>(f) | reinterpret_cast<uintptr_t>(mu ? mu : f) |
                         reinterpret_cast<uintptr_t>(qin ? qin : reinterpret_cast<const float2*>(f))) &
                        15u) == 0;
  const int vec = (g.n[2] % 4 == 0 && g.n[2] >= TXA && g.n[1] >= TY && g.n[0] >= Tile<ZB>::TZ && aligned) ? 1 : 0;
  note_launches(1);
  kern<<<nb, kTileThreads, sm, st>>>(f, mu, disp, out, g.n[0], g.n[1], g.n[2], ht, vec, NF == 2 ? qin : nullptr,
                                     NF == 2 ? qout : nullptr);
  return cudaGetLastError();
}

// Brick depths the setup autotuner chooses from (Grid::sl_bz for the state steps, sl_bz_adj for the
// adjoint steps); every depth gives the same values.
template <int MODE>
cudaError_t launch_mode(const Grid& g, const float* f, const float* mu, const float* disp, float* out, float ht,
                        const float2* qin, float2* qout, cudaStream_t st) {
  switch (MODE >= 2 ? g.sl_bz_adj : g.sl_bz) {
    case 4: return launch_mode_zb<MODE, 4>(g, f, mu, disp, out, ht, qin, qout, st);
    case 12: return launch_mode_zb<MODE, 12>(g, f, mu, disp, out, ht, qin, qout, st);
    default: return launch_mode_zb<MODE, 8>(g, f, mu, disp, out, ht, qin, qout, st);
  }
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
                           const float* mu, float* out, float ht, cudaStream_t st, const float2* qin, float2* qout) {
  if (!adjoint) {
    return continuity ? launch_mode<1>(g, f, mu, disp, out, ht, qin, qout, st)
                      : launch_mode<0>(g, f, mu, disp, out, ht, qin, qout, st);
  }
  return continuity ? launch_mode<3>(g, f, mu, disp, out, ht, qin, qout, st)
                    : launch_mode<2>(g, f, mu, disp, out, ht, qin, qout, st);
}

}  // namespace ga
