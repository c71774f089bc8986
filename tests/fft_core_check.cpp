// CPU check of the CUDA library's Stockham FFT core (compiled with g++; no GPU needed).
// For each length N it runs every stage of the plan over all butterflies in sequence (a
// sequential loop gives the same result as the parallel stage, which has no intra-stage
// dependence) and compares against a direct O(N^2) DFT evaluated in long double.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <string>
#include <vector>
#include "../paper_2510_08782_gb300/csrc/fft_core.cuh"

using namespace ga;

template <typename T, int PS>
double check(int N, unsigned seed) {
  FftPlan plan;
  if (!make_plan(N, &plan)) return -1.0;
  const int NP = fpad<PS>(N) + 1;
  std::vector<cx<T>> a(NP), b(NP), tw(N);
  for (int m = 0; m < N; ++m) {
    long double ang = -2.0L * 3.14159265358979323846264338327950288L * m / N;
    tw[m] = mk<T>((T)std::cos(ang), (T)std::sin(ang));
  }
  srand(seed);
  std::vector<long double> xr(N), xi(N);
  for (int j = 0; j < N; ++j) {
    xr[j] = (long double)rand() / RAND_MAX - 0.5L;
    xi[j] = (long double)rand() / RAND_MAX - 0.5L;
    a[fpad<PS>(j)] = mk<T>((T)xr[j], (T)xi[j]);
  }
  cx<T>* in = a.data();
  cx<T>* out = b.data();
  int Ns = 1;
  for (int s = 0; s < plan.ns; ++s) {
    int R = plan.radix[s];
    for (int j = 0; j < N / R; ++j) stockham_butterfly<T, PS>(in, out, j, N, R, Ns, tw.data());
    cx<T>* t = in; in = out; out = t;
    Ns *= R;
  }
  double err = 0.0, ref = 0.0;
  for (int k = 0; k < N; ++k) {
    long double sr = 0, si = 0;
    for (int j = 0; j < N; ++j) {
      long double ang = -2.0L * 3.14159265358979323846264338327950288L * (long double)((long long)j * k % N) / N;
      long double c = std::cos(ang), s = std::sin(ang);
      sr += xr[j] * c - xi[j] * s;
      si += xr[j] * s + xi[j] * c;
    }
    double dr = (double)(in[fpad<PS>(k)].x - sr), di = (double)(in[fpad<PS>(k)].y - si);
    err += dr * dr + di * di;
    ref += (double)(sr * sr + si * si);
  }
  return std::sqrt(err / ref);
}

// The compile-time plans used by the CUDA kernels for the common lengths (radix 16 included).
template <typename T, int N, int Ns, int MAXR, int PS>
void ct_stages(cx<T>*& in, cx<T>*& out, const cx<T>* tw) {
  if constexpr (Ns < N) {
    constexpr int R = ct_next_radix(N / Ns, MAXR);
    for (int j = 0; j < N / R; ++j) stockham_butterfly_ct<T, N, R, Ns, PS>(in, out, j, tw);
    cx<T>* t = in; in = out; out = t;
    ct_stages<T, N, Ns * R, MAXR, PS>(in, out, tw);
  }
}

template <typename T, int N, int MAXR, int PS>
double check_ct(unsigned seed) {
  const int NP = fpad<PS>(N) + 1;
  std::vector<cx<T>> a(NP), b(NP), tw(N);
  for (int m = 0; m < N; ++m) {
    long double ang = -2.0L * 3.14159265358979323846264338327950288L * m / N;
    tw[m] = mk<T>((T)std::cos(ang), (T)std::sin(ang));
  }
  srand(seed);
  std::vector<long double> xr(N), xi(N);
  for (int j = 0; j < N; ++j) {
    xr[j] = (long double)rand() / RAND_MAX - 0.5L;
    xi[j] = (long double)rand() / RAND_MAX - 0.5L;
    a[fpad<PS>(j)] = mk<T>((T)xr[j], (T)xi[j]);
  }
  cx<T>* in = a.data();
  cx<T>* out = b.data();
  ct_stages<T, N, 1, MAXR, PS>(in, out, tw.data());
  double err = 0.0, ref = 0.0;
  for (int k = 0; k < N; ++k) {
    long double sr = 0, si = 0;
    for (int j = 0; j < N; ++j) {
      long double ang = -2.0L * 3.14159265358979323846264338327950288L * (long double)((long long)j * k % N) / N;
      sr += xr[j] * std::cos(ang) - xi[j] * std::sin(ang);
      si += xr[j] * std::sin(ang) + xi[j] * std::cos(ang);
    }
    double dr = (double)(in[fpad<PS>(k)].x - sr), di = (double)(in[fpad<PS>(k)].y - si);
    err += dr * dr + di * di;
    ref += (double)(sr * sr + si * si);
  }
  return std::sqrt(err / ref);
}

template <int N> int report_ct() {
  double e[4] = {check_ct<double, N, 16, 4>(3u + N), check_ct<float, N, 16, 4>(5u + N),
                 check_ct<float, N, 8, 4>(7u + N), check_ct<float, N, 16, 0>(9u + N)};
  bool ok = e[0] < 1e-14 && e[1] < 2e-6 && e[2] < 2e-6 && e[3] < 2e-6;
  printf("compile-time N=%d fp64=%.2e fp32=%.2e fp32(radix<=8)=%.2e fp32(unpadded)=%.2e %s\n", N, e[0], e[1],
         e[2], e[3], ok ? "ok" : "FAIL");
  return ok ? 0 : 1;
}

int main(int argc, char** argv) {
  if (argc > 1 && std::string(argv[1]) == "ct") {
    return report_ct<64>() + report_ct<96>() + report_ct<128>() + report_ct<160>() + report_ct<192>() + report_ct<256>() +
           report_ct<16>() + report_ct<48>();
  }
  int fails = 0;
  for (int i = 1; i < argc; ++i) {
    int N = atoi(argv[i]);
    double ed = check<double, 0>(N, 7u + N), ef = check<float, 0>(N, 11u + N);
    double edp = check<double, 4>(N, 13u + N), efp = check<float, 4>(N, 17u + N);
    bool ok = ed >= 0 && ed < 1e-14 && ef < 2e-6 && edp < 1e-14 && efp < 2e-6;
    printf("N=%d fp64_rel_err=%.3e fp32_rel_err=%.3e %s\n", N, ed, ef, ok ? "ok" : "FAIL");
    fails += !ok;
  }
  return fails ? 1 : 0;
}
