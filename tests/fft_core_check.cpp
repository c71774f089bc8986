// CPU check of the CUDA library's Stockham FFT core (compiled with g++; no GPU needed).
// For each length N it runs every stage of the plan over all butterflies in sequence (a
// sequential loop gives the same result as the parallel stage, which has no intra-stage
// dependence) and compares against a direct O(N^2) DFT evaluated in long double.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <vector>
#include "../paper_2510_08782_gb300/csrc/fft_core.cuh"

using namespace ga;

template <typename T>
double check(int N, unsigned seed) {
  FftPlan plan;
  if (!make_plan(N, &plan)) return -1.0;
  std::vector<cx<T>> a(N), b(N), tw(N);
  for (int m = 0; m < N; ++m) {
    long double ang = -2.0L * 3.14159265358979323846264338327950288L * m / N;
    tw[m] = mk<T>((T)std::cos(ang), (T)std::sin(ang));
  }
  srand(seed);
  std::vector<long double> xr(N), xi(N);
  for (int j = 0; j < N; ++j) {
    xr[j] = (long double)rand() / RAND_MAX - 0.5L;
    xi[j] = (long double)rand() / RAND_MAX - 0.5L;
    a[j] = mk<T>((T)xr[j], (T)xi[j]);
  }
  cx<T>* in = a.data();
  cx<T>* out = b.data();
  int Ns = 1;
  for (int s = 0; s < plan.ns; ++s) {
    int R = plan.radix[s];
    for (int j = 0; j < N / R; ++j) stockham_butterfly<T>(in, out, j, N, R, Ns, tw.data());
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
    double dr = (double)(in[k].x - sr), di = (double)(in[k].y - si);
    err += dr * dr + di * di;
    ref += (double)(sr * sr + si * si);
  }
  return std::sqrt(err / ref);
}

int main(int argc, char** argv) {
  int fails = 0;
  for (int i = 1; i < argc; ++i) {
    int N = atoi(argv[i]);
    double ed = check<double>(N, 7u + N), ef = check<float>(N, 11u + N);
    bool ok = ed >= 0 && ed < 1e-14 && ef < 2e-6;
    printf("N=%d fp64_rel_err=%.3e fp32_rel_err=%.3e %s\n", N, ed, ef, ok ? "ok" : "FAIL");
    fails += !ok;
  }
  return fails ? 1 : 0;
}
