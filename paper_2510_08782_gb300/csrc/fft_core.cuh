// Mixed-radix Stockham FFT core shared by every pencil kernel (internal).
//
// The pseudo-spectral discretisation of Sec. 2.2 applies and inverts differential operators
// with FFTs. Each CUDA kernel stages a batch of pencils in shared memory and runs this
// self-sorting (Stockham) radix-2/3/4/5/8 transform on them. Stage s with radix R and span Ns
// (product of the radices already applied) maps butterfly j of every pencil as
//     v_r = x[j + r N/R] * W_N^{r (j mod Ns) N/(Ns R)},  v <- DFT_R(v),
//     y[(j - j mod Ns) R + j mod Ns + r Ns] = v_r,
// which is the classic out-of-place Stockham formulation; after the last stage the result is
// in natural order. Forward transforms use W_N = exp(-2 pi i / N); an inverse transform is done
// as conj(FFT(conj(x))). The functions are host+device so the same code is unit-tested on the CPU.
#pragma once

#include "common.cuh"

namespace ga {

// Mathematical constants of the small DFTs.
#define GA_SQRT3_2 0.86602540378443864676
#define GA_SQRT1_2 0.70710678118654752440
#define GA_C1_5 0.30901699437494742410   /* cos(2 pi / 5) */
#define GA_C2_5 (-0.80901699437494742410) /* cos(4 pi / 5) */
#define GA_S1_5 0.95105651629515357212   /* sin(2 pi / 5) */
#define GA_S2_5 0.58778525229247312917   /* sin(4 pi / 5) */

template <typename C> GA_HD void dft2(C* a) {
  C t = a[1];
  a[1] = csub(a[0], t);
  a[0] = cadd(a[0], t);
}

template <typename C> GA_HD void dft4(C* a) {
  C t0 = cadd(a[0], a[2]), t1 = csub(a[0], a[2]);
  C t2 = cadd(a[1], a[3]), t3 = cmul_negi(csub(a[1], a[3]));
  a[0] = cadd(t0, t2);
  a[2] = csub(t0, t2);
  a[1] = cadd(t1, t3);
  a[3] = csub(t1, t3);
}

template <typename T, typename C> GA_HD void dft3(C* a) {
  const T c = T(-0.5), s = T(GA_SQRT3_2);
  C sm = cadd(a[1], a[2]), df = csub(a[1], a[2]);
  C base = cadd(a[0], cscale(sm, c));
  C rot = cscale(cmul_negi(df), s);  // -i s (a1 - a2)
  a[0] = cadd(a[0], sm);
  a[1] = cadd(base, rot);
  a[2] = csub(base, rot);
}

template <typename T, typename C> GA_HD void dft5(C* a) {
  const T c1 = T(GA_C1_5), c2 = T(GA_C2_5), s1 = T(GA_S1_5), s2 = T(GA_S2_5);
  C sa = cadd(a[1], a[4]), da = csub(a[1], a[4]);
  C sb = cadd(a[2], a[3]), db = csub(a[2], a[3]);
  C r1 = cadd(a[0], cadd(cscale(sa, c1), cscale(sb, c2)));
  C r2 = cadd(a[0], cadd(cscale(sa, c2), cscale(sb, c1)));
  C i1 = cmul_negi(cadd(cscale(da, s1), cscale(db, s2)));  // -i (s1 da + s2 db)
  C i2 = cmul_negi(csub(cscale(da, s2), cscale(db, s1)));  // -i (s2 da - s1 db)
  a[0] = cadd(a[0], cadd(sa, sb));
  a[1] = cadd(r1, i1);
  a[4] = csub(r1, i1);
  a[2] = cadd(r2, i2);
  a[3] = csub(r2, i2);
}

template <typename T, typename C> GA_HD void dft8(C* a) {
  C e[4] = {a[0], a[2], a[4], a[6]};
  C o[4] = {a[1], a[3], a[5], a[7]};
  dft4(e);
  dft4(o);
  const T r = T(GA_SQRT1_2);
  // twiddles W8^k, k = 0..3: 1, (r, -r), -i, (-r, -r)
  C o1 = mk<T>((o[1].x + o[1].y) * r, (o[1].y - o[1].x) * r);
  C o2 = cmul_negi(o[2]);
  C o3 = mk<T>((o[3].y - o[3].x) * r, -(o[3].x + o[3].y) * r);
  a[0] = cadd(e[0], o[0]);
  a[4] = csub(e[0], o[0]);
  a[1] = cadd(e[1], o1);
  a[5] = csub(e[1], o1);
  a[2] = cadd(e[2], o2);
  a[6] = csub(e[2], o2);
  a[3] = cadd(e[3], o3);
  a[7] = csub(e[3], o3);
}

// 16-point DFT in registers as 4 x 4: inner DFT4s over n1 (stride 4), twiddles W16^(n2 k1), outer
// DFT4s over n2; output index k1 + 4 k2.
#define GA_C1_16 0.92387953251128675613 /* cos(pi / 8) */
#define GA_S1_16 0.38268343236508977173 /* sin(pi / 8) */
template <typename T, typename C> GA_HD void dft16(C* a) {
  C y[4][4];
  for (int n2 = 0; n2 < 4; ++n2) {
    C t[4] = {a[n2], a[4 + n2], a[8 + n2], a[12 + n2]};
    dft4(t);
    for (int k1 = 0; k1 < 4; ++k1) y[n2][k1] = t[k1];
  }
  const T c = T(GA_C1_16), s = T(GA_S1_16), r = T(GA_SQRT1_2);
  // W16^m = exp(-2 pi i m / 16) for m = n2 k1
  y[1][1] = cmul(y[1][1], mk<T>(c, -s));
  y[1][2] = cmul(y[1][2], mk<T>(r, -r));
  y[1][3] = cmul(y[1][3], mk<T>(s, -c));
  y[2][1] = cmul(y[2][1], mk<T>(r, -r));
  y[2][2] = cmul_negi(y[2][2]);
  y[2][3] = cmul(y[2][3], mk<T>(-r, -r));
  y[3][1] = cmul(y[3][1], mk<T>(s, -c));
  y[3][2] = cmul(y[3][2], mk<T>(-r, -r));
  y[3][3] = cmul(y[3][3], mk<T>(-c, s));
  for (int k1 = 0; k1 < 4; ++k1) {
    C t[4] = {y[0][k1], y[1][k1], y[2][k1], y[3][k1]};
    dft4(t);
    for (int k2 = 0; k2 < 4; ++k2) a[k1 + 4 * k2] = t[k2];
  }
}

// Shared-memory position of pencil element i: with PS > 0 one padding entry is inserted after every
// 2^PS entries, which makes the power-of-two strides of the Stockham stages odd and so free of
// bank conflicts for 8-byte (complex FP32) accesses.
template <int PS> GA_HD int fpad(int i) { return PS > 0 ? i + (i >> PS) : i; }

// One butterfly of one Stockham stage. `in`/`out` point at the start of the pencil.
template <typename T, int PS = 0>
GA_HD void stockham_butterfly(const cx<T>* in, cx<T>* out, int j, int N, int R, int Ns,
                              const cx<T>* tw) {
  const int M = N / R;
  const int k = j % Ns;
  const int tstep = k * (N / (Ns * R));
  cx<T> v[8];
  v[0] = in[fpad<PS>(j)];
  for (int r = 1; r < R; ++r) v[r] = cmul(in[fpad<PS>(j + r * M)], tw[r * tstep]);
  switch (R) {
    case 2: dft2(v); break;
    case 3: dft3<T>(v); break;
    case 4: dft4(v); break;
    case 5: dft5<T>(v); break;
    default: dft8<T>(v); break;
  }
  const int base = (j - k) * R + k;
  for (int r = 0; r < R; ++r) out[fpad<PS>(base + r * Ns)] = v[r];
}

// Compile-time variant of one stage for a fixed length N, radix R and span Ns: every index
// operation folds to constants (shifts and masks for powers of two).
#if defined(__CUDACC__)
__host__ __device__
#endif
constexpr int ct_next_radix(int rem, int maxr = 16) {
  return (maxr >= 16 && rem % 16 == 0) ? 16
                                       : (rem % 8 == 0 ? 8 : (rem % 4 == 0 ? 4 : (rem % 2 == 0 ? 2 : (rem % 3 == 0 ? 3 : 5))));
}

template <typename T, int N, int R, int Ns, int PS = 0>
GA_HD void stockham_butterfly_ct(const cx<T>* in, cx<T>* out, int j, const cx<T>* tw) {
  constexpr int M = N / R;
  const int k = j % Ns;
  const int tstep = k * (N / (Ns * R));
  cx<T> v[R];
  v[0] = in[fpad<PS>(j)];
  if constexpr (Ns == 1) {  // first stage: every twiddle is 1
#pragma unroll
    for (int r = 1; r < R; ++r) v[r] = in[fpad<PS>(j + r * M)];
  } else {
#pragma unroll
    for (int r = 1; r < R; ++r) v[r] = cmul(in[fpad<PS>(j + r * M)], tw[r * tstep]);
  }
  if constexpr (R == 2) dft2(v);
  else if constexpr (R == 3) dft3<T>(v);
  else if constexpr (R == 4) dft4(v);
  else if constexpr (R == 5) dft5<T>(v);
  else if constexpr (R == 16) dft16<T>(v);
  else dft8<T>(v);
  const int base = (j - k) * R + k;
#pragma unroll
  for (int r = 0; r < R; ++r) out[fpad<PS>(base + r * Ns)] = v[r];
}

// Host: factor N into radices (8s first for powers of two, then 4/2, 3, 5). Returns false if N
// has a prime factor other than 2, 3, 5 or if N < 1.
inline bool make_plan(int N, FftPlan* p) {
  if (N < 1) return false;
  p->n = N;
  p->ns = 0;
  int m = N;
  int twos = 0;
  while (m % 2 == 0) { m /= 2; ++twos; }
  while (twos >= 3) { p->radix[p->ns++] = 8; twos -= 3; }
  if (twos == 2) p->radix[p->ns++] = 4;
  if (twos == 1) p->radix[p->ns++] = 2;
  while (m % 3 == 0) { m /= 3; p->radix[p->ns++] = 3; }
  while (m % 5 == 0) { m /= 5; p->radix[p->ns++] = 5; }
  return m == 1 && p->ns < 24;
}

}  // namespace ga
