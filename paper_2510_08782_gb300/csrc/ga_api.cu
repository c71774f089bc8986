// Runtime behind the C ABI of include/ga.h and include/ga_ops.h.
//
// One context owns every device buffer of one problem and orders its work on one stream (the body
// force's derivative passes run on a second stream of the context, joined by events). The
// gradient evaluation (Eq. (3)) runs as: the regulariser value 1/2 <v, w> with w = alpha L v (carried
// by the solver with v; formed by the transform for a caller's v), mu = div v by 1D derivative
// passes, RK2 departure points, n_t state steps (all states or checkpoints every K), mismatch and
// terminal adjoint value, then backwards in time the body force h_t w_j lambda_j grad m_j (one fused
// FFT-derivative pass per axis) and the adjoint step, then g = (P) b + w in real space and, for the
// solver, s = -(alpha L)^{-1} (P) g and alpha L s by one transform of g.
// The solver (Alg. 3) drives the line search from the host: each Armijo trial is a state solve whose
// FP64 objective is read back; the window inner products, the Gram update, the least-squares solve
// and the combination run on the device.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <array>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <type_traits>
#include <vector>

#include "../../include/ga.h"
#include "../../include/ga_ops.h"
#include "fft_core.cuh"
#include "kernels.h"

using namespace ga;

#include <atomic>

namespace ga {
static std::atomic<long long> g_launches{0};
static thread_local long long t_launches = 0;  // this thread's share (kernel counts of a capture)
void note_launches(int n) {
  g_launches.fetch_add(n, std::memory_order_relaxed);
  t_launches += n;
}
}  // namespace ga

namespace {

constexpr int kNumRes = 128;                // device FP64 result slots
constexpr int kResDots = 16;                // first slot of the window inner products
constexpr int kResLsq = kResDots + kMaxDots;  // least-squares diagnostics

struct Fail {
  ga_status st;
};

}  // namespace

struct EngineBase {
  virtual ~EngineBase() {}
};

template <typename T> struct Engine;

struct ga_ctx {
  ga_problem_desc desc;
  ga_solver_opts opts;
  cudaStream_t st = nullptr;
  std::string err;
  ga_stats stats;
  int prec = 0;
  Engine<float>* ef = nullptr;
  Engine<double>* ed = nullptr;
};

namespace {

void set_err(ga_ctx* c, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
}

}  // namespace

template <typename T> struct Engine : EngineBase {
  ga_ctx* ctx;
  Grid g;
  int dim, nt, model, s, K;
  double alpha, ht, hd;
  long long nv, vl;
  cudaStream_t st;
  FftTables<T> ft;
  cx<T>* twd[3] = {nullptr, nullptr, nullptr};  // the device twiddle tables ft.tw points at
  cx<T>* qp[2] = {nullptr, nullptr};            // (pi, pi mu) pairs of the continuity state chain
  const T* q_src = nullptr;
  int q_idx = 0;
  cx<T>* ap[2] = {nullptr, nullptr};            // (lambda, lambda mu) pairs of the advection adjoint chain
  const T* a_src = nullptr;
  int a_idx = 0;
  std::vector<void*> allocs;
  void* pinned = nullptr;
  double* hres = nullptr;

  T *m0 = nullptr, *m1 = nullptr, *xm = nullptr, *xp = nullptr, *mu = nullptr;
  // adjoint states: a ring, so the adjoint steps run ahead of the body-force passes that read them
  static constexpr int kLamRing = 6;
  T* lam[kLamRing] = {};
  T *body = nullptr, *tmp[2] = {nullptr, nullptr};
  T* wtmp = nullptr;  // alpha L v for calls that do not carry it
  // recomputed checkpoint segments: two buffers, so a recompute does not wait for the passes that
  // read the previous segment; seg_base[b] is the first state index of the segment buffer b holds
  T *states = nullptr, *seg[2] = {nullptr, nullptr}, *io_a = nullptr, *io_b = nullptr;
  int nslots = 0, seg_base[2] = {-1, -1}, seg_next = 0;
  // The body force's derivative passes run on st2, overlapped with the adjoint steps and recomputed
  // state steps on st. Group g (the passes of one trapezoid pair) ends with bf_ev[g] on st2; a buffer
  // that group read is written again on st only after st has waited for bf_ev[g].
  cudaStream_t st2 = nullptr;
  cudaEvent_t bf_fork = nullptr, bf_join = nullptr;
  std::vector<cudaEvent_t> bf_ev;
  int lam_reader[kLamRing] = {}, seg_reader[2] = {-1, -1}, bf_waited = -1;
  bool bf_active = false;
  cx<T> *vh = nullptr, *bh = nullptr;
  double *dpart = nullptr, *dres = nullptr, *dM = nullptr, *dbeta = nullptr;

  // solver state
  int W1 = 1;
  std::vector<T*> vfree, gfree;
  std::deque<std::pair<T*, T*>> win;  // (v, g), newest first
  T* S = nullptr;                      // preconditioned direction at the current iterate
  bool s_valid = false, started = false;
  int k = 0;
  double g0inf = 0.0, J = 0.0, mis = 0.0, rho_mem = 1.0;
  cudaEvent_t ev[2] = {nullptr, nullptr};

  // profiling of one kernel class with events (see ga_prof_start)
  int prof_class = -1;
  std::vector<cudaEvent_t> prof_ev;
  int prof_used = 0;
  double prof_ms = 0.0;
  long long prof_launches = 0;

  ~Engine() override {
    for (void* p : allocs) cudaFree(p);
    if (pinned) cudaFreeHost(pinned);
    if (ev[0]) cudaEventDestroy(ev[0]);
    if (ev[1]) cudaEventDestroy(ev[1]);
    for (auto e : prof_ev) cudaEventDestroy(e);
    for (auto e : bf_ev) cudaEventDestroy(e);
    if (bf_fork) cudaEventDestroy(bf_fork);
    if (bf_join) cudaEventDestroy(bf_join);
    if (st2) cudaStreamDestroy(st2);
    for (auto ge : gexec)
      if (ge) cudaGraphExecDestroy(ge);
    if (gst) cudaStreamDestroy(gst);
    if (rexec) cudaGraphExecDestroy(rexec);
    for (auto cs : cap)
      if (cs) cudaStreamDestroy(cs);
    if (hctl) cudaFreeHost(hctl);
  }

  void ck(cudaError_t e, const char* what) {
    if (e != cudaSuccess) {
      set_err(ctx, "%s: %s", what, cudaGetErrorString(e));
      throw Fail{e == cudaErrorMemoryAllocation ? GA_ERR_NOMEM : GA_ERR_CUDA};
    }
  }
  template <typename U> U* dalloc(long long count) {
    void* p = nullptr;
    if (count < 1) count = 1;
    cudaError_t e = cudaMalloc(&p, sizeof(U) * (size_t)count);
    if (e != cudaSuccess) {
      cudaGetLastError();
      set_err(ctx, "cudaMalloc of %lld bytes failed: %s", (long long)(sizeof(U) * count), cudaGetErrorString(e));
      throw Fail{GA_ERR_NOMEM};
    }
    allocs.push_back(p);
    return static_cast<U*>(p);
  }

  // Sizes that follow from the descriptor and the solver options (shared by init and the workspace
  // planner, ga_workspace_bytes).
  void derive(const ga_problem_desc& d, const ga_solver_opts& o) {
    dim = d.dim;
    nt = d.nt;
    model = d.model;
    s = d.reg_order;
    alpha = d.alpha;
    K = d.ckpt_every;
    g.dim = dim;
    if (dim == 3) {
      g.n[0] = d.n[0];
      g.n[1] = d.n[1];
      g.n[2] = d.n[2];
    } else {
      g.n[0] = 1;
      g.n[1] = d.n[0];
      g.n[2] = d.n[1];
    }
    g.n2h = g.n[2] / 2 + 1;
    g.nvox = (long long)g.n[0] * g.n[1] * g.n[2];
    g.nhalf = (long long)g.n[0] * g.n[1] * g.n2h;
    nv = g.nvox;
    vl = nv * dim;
    ht = 1.0 / nt;
    hd = 1.0;
    for (int a = 3 - dim; a < 3; ++a) hd *= 2.0 * M_PI / g.n[a];
    nslots = (K == 0) ? nt : (nt / K + (nt % K != 0 ? 1 : 0));
    // solver pools: window (w+1) + trial q + one more, for iterates and gradients. An iterate buffer
    // holds v in [0, vl) and w = alpha L v in [vl, 2 vl); S holds s and alpha L s the same way.
    W1 = o.window + 1;
    resident = o.graphs == 2;
    graphs = o.graphs == 1;
  }

  // Every device buffer a context holds from ga_setup on, in allocation order: al(pointer, element
  // count). The only later allocation is the discretise-then-optimise gradient's buffer (one vector
  // field, on its first use).
  template <class A> void layout(A&& al) {
    for (int a = 0; a < 3; ++a) al(twd[a], (long long)g.n[a]);  // twiddle tables exp(-2 pi i m / n_a)
    al(m0, nv);
    al(m1, nv);
    al(xm, vl);
    al(xp, vl);
    al(mu, nv);
    for (int i = 0; i < kLamRing; ++i) al(lam[i], nv);
    al(tmp[0], nv);
    al(tmp[1], nv);
    al(body, vl);
    al(io_a, vl);
    al(io_b, vl);
    al(states, (long long)nslots * nv);
    if (K > 1) {
      al(seg[0], (long long)(K - 1) * nv);
      al(seg[1], (long long)(K - 1) * nv);
    }
    al(vh, g.nhalf * dim);
    al(bh, g.nhalf * dim);
    al(dpart, (long long)kMaxDots * kRedBlocks);
    al(dres, (long long)kNumRes);
    if (resident) {  // the same memory as the pools, in fixed roles (see the device-driven solve below)
      al(VC, 2 * vl);
      al(Q, 2 * vl);
      al(GC, vl);
      al(GQ, vl);
      al(RV, (long long)W1 * 2 * vl);
      al(RG, (long long)W1 * vl);
      al(dctl, 1LL);
    } else {
      for (int i = 0; i < W1 + 2; ++i) {
        T* pv = nullptr;
        T* pg = nullptr;
        al(pv, 2 * vl);
        al(pg, vl);
        vfree.push_back(pv);
        gfree.push_back(pg);
      }
    }
    al(S, 2 * vl);
    al(wtmp, vl);
    if (graphs) {
      al(gin, 2 * vl);
      al(gbuf, vl);
    }
    al(dM, (long long)W1 * W1);
    al(dbeta, (long long)kMaxWin + 4);
    if (std::is_same<T, float>::value && dim == 3 && model == GA_MODEL_CONTINUITY) {
      al(qp[0], nv);
      al(qp[1], nv);
    }
    if (std::is_same<T, float>::value && dim == 3 && model != GA_MODEL_CONTINUITY) {
      al(ap[0], nv);
      al(ap[1], nv);
    }
  }

  void init(ga_ctx* c, const void* hm0, const void* hm1, int mem) {
    ctx = c;
    st = c->st;
    derive(c->desc, c->opts);
    ck(cudaEventCreate(&ev[0]), "cudaEventCreate");
    ck(cudaEventCreate(&ev[1]), "cudaEventCreate");
    ck(cudaStreamCreateWithFlags(&st2, cudaStreamNonBlocking), "body-force stream");
    ck(cudaEventCreateWithFlags(&bf_fork, cudaEventDisableTiming), "cudaEventCreate");
    ck(cudaEventCreateWithFlags(&bf_join, cudaEventDisableTiming), "cudaEventCreate");
    bf_ev.resize(nt / 2 + 2);
    for (auto& e : bf_ev) ck(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "cudaEventCreate");
    layout([&](auto*& p, long long count) {
      using U = std::remove_reference_t<decltype(*p)>;
      p = dalloc<U>(count);
    });

    // FFT plans and twiddle tables per internal axis
    for (int a = 0; a < 3; ++a) {
      make_plan(g.n[a], &ft.plan[a]);
      const int L = g.n[a];
      std::vector<cx<T>> tw(L);
      for (int m = 0; m < L; ++m) {
        // angle -2 pi m / L, reduced to the first octants for accuracy
        const long double ang = -2.0L * 3.14159265358979323846264338327950288L * (long double)m / L;
        tw[m] = mk<T>((T)cosl(ang), (T)sinl(ang));
      }
      ck(cudaMemcpy(twd[a], tw.data(), sizeof(cx<T>) * L, cudaMemcpyHostToDevice), "twiddle upload");
      ft.tw[a] = twd[a];
    }

    const cudaMemcpyKind kind = mem == GA_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    ck(cudaMemcpyAsync(m0, hm0, sizeof(T) * nv, kind, st), "copy m0");
    ck(cudaMemcpyAsync(m1, hm1, sizeof(T) * nv, kind, st), "copy m1");
    ck(cudaMallocHost(&pinned, sizeof(double) * kNumRes), "cudaMallocHost");
    hres = static_cast<double*>(pinned);
    if (resident) {
      void* hp = nullptr;
      ck(cudaMallocHost(&hp, sizeof(ResCtl)), "cudaMallocHost");
      hctl = static_cast<ResCtl*>(hp);
      std::memset(hctl, 0, sizeof(ResCtl));
      for (auto& cs : cap) ck(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "capture stream");
    }
    if (graphs && (st == nullptr || st == cudaStreamLegacy || st == cudaStreamPerThread))
      ck(cudaStreamCreate(&gst), "capture stream");
    ck(cudaMemsetAsync(dM, 0, sizeof(double) * W1 * W1, st), "memset");
    autotune_tiles();
    ck(cudaStreamSynchronize(st), "setup sync");
  }

  // ---- tile autotuner --------------------------------------------------------------------------
  // The FFT-derivative passes take their tile shape, the number of complex pencils a CTA transforms,
  // from timing: for each axis, and separately for the one-field passes (div v) and the two-time-step
  // passes of the body force, the default, its half and its double are run on this context's own fields
  // (m0 differentiated, times m1, accumulated into a scratch field) and the fastest is kept. Choices
  // are cached per (precision, grid) for the process. Each pencil is transformed on its own, so no
  // result depends on the choice.
  void autotune_tiles() {
    static std::mutex mu;
    static std::map<std::vector<int>, std::array<int, 8>> cache;
    const std::vector<int> key = {(int)sizeof(T), g.n[0], g.n[1], g.n[2], model};
    {
      std::lock_guard<std::mutex> lk(mu);
      auto it = cache.find(key);
      if (it != cache.end()) {
        for (int a = 0; a < 3; ++a) {
          ft.deriv_pencils[a] = it->second[a];
          ft.pair_pencils[a] = it->second[3 + a];
        }
        g.sl_bz = it->second[6];
        g.sl_bz_adj = it->second[7];
        return;
      }
    }
    std::array<int, 8> best = {0, 0, 0, 0, 0, 0, 8, 8};
    for (int pair = 0; pair < 2; ++pair) {
      for (int a = 3 - dim; a < 3; ++a) {
        const int L = g.n[a];
        if (L == 1) continue;
        int* slot = pair ? &ft.pair_pencils[a] : &ft.deriv_pencils[a];
        if (L == kRegFftLen) {  // the register-resident transform: a fixed tile, nothing to tune
          *slot = kRegFftPencils;
          best[3 * pair + a] = kRegFftPencils;
          continue;
        }
        const int b0 = deriv_default_pencils<T>(L);
        float best_ms = 0.f;
        int choice = 0;
        for (int cand : {b0, b0 / 2, 2 * b0}) {
          if (!deriv_pencils_fit<T>(L, cand)) continue;
          *slot = cand;
          auto pass = [&](bool acc) {
            if (pair) ck(launch_deriv_pair<T>(g, ft, a, m0, m1, T(1), m1, m0, T(1), tmp[0], acc, st), "tuning pass");
            else ck(launch_deriv<T>(g, ft, a, m0, m1, tmp[0], T(1), acc, st), "tuning pass");
          };
          pass(false);  // loads the kernel
          ck(cudaEventRecord(ev[0], st), "event");
          for (int r = 0; r < 3; ++r) pass(true);
          ck(cudaEventRecord(ev[1], st), "event");
          ck(cudaEventSynchronize(ev[1]), "event sync");
          float ms = 0.f;
          ck(cudaEventElapsedTime(&ms, ev[0], ev[1]), "event time");
          if (choice == 0 || ms < best_ms) {
            choice = cand;
            best_ms = ms;
          }
        }
        *slot = choice;
        best[3 * pair + a] = choice;
      }
    }
    // Brick depths of the FP32 3D transport steps, at zero displacement (the shared-memory gather every
    // in-halo voxel takes): for the state steps, chained steps of this model (a step fed by the previous
    // one, as in a sweep); for the adjoint steps, adjoint steps. The two are chosen separately.
    if (std::is_same<T, float>::value && dim == 3) {
      ck(cudaMemsetAsync(xm, 0, sizeof(T) * vl, st), "memset");
      ck(cudaMemsetAsync(xp, 0, sizeof(T) * vl, st), "memset");
      ck(cudaMemsetAsync(this->mu, 0, sizeof(T) * nv, st), "memset");
      auto timed = [&](auto&& run) {
        run();  // loads the kernels
        ck(cudaEventRecord(ev[0], st), "event");
        for (int r = 0; r < 3; ++r) run();
        ck(cudaEventRecord(ev[1], st), "event");
        ck(cudaEventSynchronize(ev[1]), "event sync");
        float ms = 0.f;
        ck(cudaEventElapsedTime(&ms, ev[0], ev[1]), "event time");
        return ms;
      };
      float best_f = 0.f, best_a = 0.f;
      int choice_f = 0, choice_a = 0;
      for (int zb : kSlDepths) {
        g.sl_bz = zb;
        chain_reset();
        sl_forward(m0, tmp[0]);
        const float mf = timed([&] {
          sl_forward(tmp[0], tmp[1]);
          sl_forward(tmp[1], tmp[0]);
        });
        if (choice_f == 0 || mf < best_f) {
          choice_f = zb;
          best_f = mf;
        }
        g.sl_bz_adj = zb;
        adjoint_chain_reset();
        const float ma = timed([&] {
          sl_adjoint(m1, tmp[1]);
          sl_adjoint(m0, tmp[1]);
        });
        if (choice_a == 0 || ma < best_a) {
          choice_a = zb;
          best_a = ma;
        }
      }
      g.sl_bz = choice_f;
      g.sl_bz_adj = choice_a;
      best[6] = choice_f;
      best[7] = choice_a;
    }
    std::lock_guard<std::mutex> lk(mu);
    cache.emplace(key, best);
  }

  // ---- profiling hooks ------------------------------------------------------------------------
  enum { PROF_SL_FWD = 0, PROF_DERIV = 1, PROF_FFT = 2, PROF_SL_ADJ = 3, PROF_DERIV_PAIR = 4 };
  void prof_begin(int cls) { prof_begin(cls, st); }
  void prof_end(int cls) { prof_end(cls, st); }
  void prof_begin(int cls, cudaStream_t s) {
    if (prof_class != cls) return;
    if (prof_used + 2 > (int)prof_ev.size()) prof_flush();
    ck(cudaEventRecord(prof_ev[prof_used], s), "cudaEventRecord");
  }
  void prof_end(int cls, cudaStream_t s) {
    if (prof_class != cls) return;
    ck(cudaEventRecord(prof_ev[prof_used + 1], s), "cudaEventRecord");
    prof_used += 2;
    ++prof_launches;
  }
  void prof_flush() {
    if (prof_used == 0) return;
    ck(cudaEventSynchronize(prof_ev[prof_used - 1]), "cudaEventSynchronize");
    for (int i = 0; i < prof_used; i += 2) {
      float ms = 0.f;
      ck(cudaEventElapsedTime(&ms, prof_ev[i], prof_ev[i + 1]), "cudaEventElapsedTime");
      prof_ms += ms;
    }
    prof_used = 0;
  }

  // ---- building blocks --------------------------------------------------------------------------
  const T* slot(int j) const {
    if (j == 0) return m0;
    if (K == 0) return states + (long long)(j - 1) * nv;
    if (j % K == 0) return states + (long long)(j / K - 1) * nv;
    return states + (long long)(nt / K) * nv;  // the final state when K does not divide n_t
  }
  bool stored(int j) const { return K == 0 || j % K == 0 || j == nt; }

  // One state step. Continuity steps of FP32 3D grids also write the pairs (pi_{j+1}, pi_{j+1} mu) into
  // one of two chain buffers qp, and a step whose input is the previous step's output stages those pairs
  // as they are (no interleaving pass). q_src names the state whose pairs qp[q_idx] holds; every chain
  // of steps starts with chain_reset(), so a chain never reads pairs of a state it did not write.
  void chain_reset() {
    q_src = nullptr;
    q_idx = 0;
  }
  void sl_forward(const T* src, T* dst) {
    cx<T>* qin = nullptr;
    cx<T>* qout = nullptr;
    if (qp[0]) {
      if (src != nullptr && src == q_src) {
        qin = qp[q_idx];
        q_idx ^= 1;
      }
      qout = qp[q_idx];
      q_src = dst;
    }
    prof_begin(PROF_SL_FWD);
    ck(launch_sl_forward<T>(g, model == GA_MODEL_CONTINUITY, src, xm, mu, dst, (T)ht, st, qin, qout), "sl_forward");
    prof_end(PROF_SL_FWD);
  }
  // One adjoint step. Advection adjoint steps (two fields, lambda and lambda mu) of FP32 3D grids chain
  // their pairs the same way through ap, with their own chain state (a backward sweep interleaves
  // recomputed state steps).
  void adjoint_chain_reset() {
    a_src = nullptr;
    a_idx = 0;
  }
  void sl_adjoint(const T* src, T* dst) {
    cx<T>* qin = nullptr;
    cx<T>* qout = nullptr;
    if (ap[0]) {
      if (src != nullptr && src == a_src) {
        qin = ap[a_idx];
        a_idx ^= 1;
      }
      qout = ap[a_idx];
      a_src = dst;
    }
    prof_begin(PROF_SL_ADJ);
    ck(launch_sl_adjoint<T>(g, model == GA_MODEL_CONTINUITY, src, xp, mu, dst, (T)ht, st, qin, qout), "sl_adjoint");
    prof_end(PROF_SL_ADJ);
  }
  void deriv(int axis, const T* f, const T* mult, T* out, double coef, bool acc) { deriv(axis, f, mult, out, coef, acc, st); }
  void deriv(int axis, const T* f, const T* mult, T* out, double coef, bool acc, cudaStream_t s) {
    prof_begin(PROF_DERIV, s);
    ck(launch_deriv<T>(g, ft, axis, f, mult, out, (T)coef, acc, s), "deriv");
    prof_end(PROF_DERIV, s);
  }
  // out += coef mult d f + coef2 mult2 d f2 along `axis` (two time steps of the body force), on stream s
  void deriv_pair(int axis, const T* f, const T* mult, double coef, const T* f2, const T* mult2, double coef2,
                  T* out, cudaStream_t s) {
    prof_begin(PROF_DERIV_PAIR, s);
    ck(launch_deriv_pair<T>(g, ft, axis, f, mult, (T)coef, f2, mult2, (T)coef2, out, true, s), "deriv pair");
    prof_end(PROF_DERIV_PAIR, s);
  }
  void r2c(const T* f, cx<T>* fh) {
    prof_begin(PROF_FFT);
    ck(launch_r2c<T>(g, ft, f, fh, st), "r2c");
    prof_end(PROF_FFT);
  }
  void c2r(cx<T>* fh, T* f) {
    prof_begin(PROF_FFT);
    ck(launch_c2r<T>(g, ft, fh, f, st), "c2r");
    prof_end(PROF_FFT);
  }

  void compute_mu(const T* v) {
    for (int c = 0; c < dim; ++c) deriv(g.axis_of(c), v + c * nv, nullptr, mu, 1.0, c > 0);
  }
  bool needs_mu_forward() const { return model == GA_MODEL_CONTINUITY; }
  bool needs_mu_adjoint() const { return model != GA_MODEL_CONTINUITY; }

  // F v into vh and the regulariser sum into dres[slot]
  // w = alpha L v by the transform (Sec. 2.2): used where w is not carried along with v.
  void apply_alphaL(const T* v, T* w) {
    for (int c = 0; c < dim; ++c) r2c(v + c * nv, vh + c * g.nhalf);
    SpecArgs sa{SPEC_APPLY_ALPHA_L, s, alpha, 0};
    ck(launch_spectral<T>(g, sa, vh, st), "spectral alpha L");
    for (int c = 0; c < dim; ++c) c2r(vh + c * g.nhalf, w + c * nv);
  }
  // sum_x v . w into dres[slot]; the regulariser (alpha/2) <v, L v> is h^d/2 times it for w = alpha L v.
  void reg_dot(const T* v, const T* w, int slot) {
    const T* bl[1] = {w};
    ck(launch_dots<T>(v, bl, 1, vl, dpart, dres + slot, st), "regulariser dot");
  }
  double reg_value(double raw) const { return 0.5 * hd * raw; }

  // s = -(alpha L)^{-1} (P) g (Eq. (9)) into sout and, when tout != nullptr, t = alpha L s into tout.
  // Advection/continuity: alpha L^ s^ = -g^ for k != 0 and 0 at k = 0, so t = -(g - mean g) in real
  // space. Incompressible: t^ = alpha L^ s^ by the transform.
  void precond_into(const T* gin, T* sout, T* tout) {
    for (int c = 0; c < dim; ++c) r2c(gin + c * nv, bh + c * g.nhalf);
    const bool inc = model == GA_MODEL_INCOMPRESSIBLE;
    if (tout && !inc) ck(launch_neg_centered<T>(g, gin, bh, tout, st), "alpha L s");
    SpecArgs sa{SPEC_PRECOND, s, alpha, inc ? 1 : 0};
    ck(launch_spectral<T>(g, sa, bh, st), "spectral precond");
    if (tout && inc) {
      ck(cudaMemcpyAsync(vh, bh, sizeof(cx<T>) * g.nhalf * dim, cudaMemcpyDeviceToDevice, st), "copy s^");
      SpecArgs sl{SPEC_APPLY_ALPHA_L, s, alpha, 0};
      ck(launch_spectral<T>(g, sl, vh, st), "spectral alpha L s");
      for (int c = 0; c < dim; ++c) c2r(vh + c * g.nhalf, tout + c * nv);
    }
    for (int c = 0; c < dim; ++c) c2r(bh + c * g.nhalf, sout + c * nv);
  }

  // State solve keeping only the final state; returns pointer to m(1).
  const T* forward_final(const T* v) {
    ck(launch_departure<T>(g, v, xm, xp, (T)ht, st, /*both=*/0), "departure");
    chain_reset();
    const T* cur = m0;
    for (int j = 0; j < nt; ++j) {
      T* dst = tmp[(j + 1) & 1];
      sl_forward(cur, dst);
      cur = dst;
    }
    return cur;
  }

  // First state index of the last checkpoint segment that has unstored states (they are recomputed in
  // the backward sweep), or -1 when there is none.
  int last_segment() const {
    if (K <= 1 || (nt - 1) % K == 0) return -1;
    return ((nt - 1) / K) * K;
  }
  // State solve storing the checkpoints. The unstored states of the last segment go straight to the
  // segment buffer, where the backward sweep, which starts there, finds them: that segment is never
  // recomputed.
  void forward_all() {
    chain_reset();
    const T* cur = m0;
    const int jl = last_segment();
    for (int j = 0; j < nt; ++j) {
      T* dst;
      if (stored(j + 1)) dst = const_cast<T*>(slot(j + 1));
      else if (jl >= 0 && j + 1 > jl) dst = seg[0] + (long long)(j - jl) * nv;
      else dst = tmp[(j + 1) & 1];
      sl_forward(cur, dst);
      cur = dst;
    }
    segs_after_forward();
  }
  // The segment buffers as forward_all leaves them: the last segment (if any) in seg[0].
  void segs_after_forward() {
    seg_base[0] = last_segment();
    seg_base[1] = -1;
    seg_next = 1;
  }

  // State j: a stored state, or one of a recomputed segment. A segment is recomputed from its
  // checkpoint into the segment buffer used less recently, once the body-force passes that read that
  // buffer's segment are done.
  const T* state(int j) {
    if (stored(j)) return slot(j);
    const int js = (j / K) * K;
    for (int b = 0; b < 2; ++b)
      if (seg_base[b] == js) return seg[b] + (long long)(j - js - 1) * nv;
    const int b = seg_next;
    seg_next ^= 1;
    bf_wait(seg_reader[b]);
    seg_reader[b] = -1;
    chain_reset();
    const T* cur = slot(js);
    const int last = (js + K - 1 < nt - 1) ? js + K - 1 : nt - 1;
    for (int i = js + 1; i <= last; ++i) {
      T* dst = seg[b] + (long long)(i - js - 1) * nv;
      sl_forward(cur, dst);
      cur = dst;
    }
    seg_base[b] = js;
    return seg[b] + (long long)(j - js - 1) * nv;
  }
  // st waits until body-force group grp (and every earlier one) is done on st2.
  void bf_wait(int grp) {
    if (grp <= bf_waited) return;
    ck(cudaStreamWaitEvent(st, bf_ev[grp], 0), "wait body-force passes");
    bf_waited = grp;
  }

  void issue_results(int count) {
    if (!host_results) return;  // recorded into the device-driven solve's graph: results stay on the device
    ck(cudaMemcpyAsync(hres, dres, sizeof(double) * count, cudaMemcpyDeviceToHost, st), "result copy");
  }
  bool host_results = true;
  void wait_results() {
    ck(cudaStreamSynchronize(st), "sync");
    prof_flush();
  }
  void read_results(int count) {
    issue_results(count);
    wait_results();
  }

  // ---- CUDA graphs of the solver's evaluations (ga_solver_opts.graphs) ---------------------------
  // The evaluations the solver repeats run on fixed buffers: v and w are copied into gin, the gradient
  // comes out of gbuf and s goes to S. Variant id's first call runs eagerly (it loads every kernel and
  // sets every launch attribute), the second is captured into a graph, later calls replay it.
  enum { G_OBJ = 0, G_OBJ_KEEP = 1, G_GRAD = 2, G_GRAD_REUSE = 3, G_GRAD_S = 4, G_GRAD_REUSE_S = 5, G_NUM = 6 };
  bool graphs = false;
  // A default stream cannot be captured: graphs are then captured and replayed on a private blocking
  // stream, which orders itself against the legacy default stream in both directions.
  cudaStream_t gst = nullptr;
  T* gin = nullptr;
  T* gbuf = nullptr;
  cudaGraphExec_t gexec[G_NUM] = {};
  long long gkernels[G_NUM] = {};
  int gcalls[G_NUM] = {};

  template <typename F> void run_variant(int id, F&& enqueue) {
    if (gcalls[id]++ == 0) {
      enqueue();
      return;
    }
    cudaStream_t cs = gst ? gst : st;
    if (!gexec[id]) {
      const long long c0 = t_launches;
      ck(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal), "begin capture");
      cudaStream_t saved = st;
      st = cs;  // every launch of enqueue() goes to the captured stream
      cudaGraph_t graph = nullptr;
      try {
        enqueue();
      } catch (...) {
        st = saved;
        cudaStreamEndCapture(cs, &graph);
        if (graph) cudaGraphDestroy(graph);
        throw;
      }
      st = saved;
      ck(cudaStreamEndCapture(cs, &graph), "end capture");
      const cudaError_t e = cudaGraphInstantiate(&gexec[id], graph, 0);
      cudaGraphDestroy(graph);
      ck(e, "graph instantiate");
      gkernels[id] = t_launches - c0;
      note_launches((int)-gkernels[id]);  // recorded, not launched
    }
    ck(cudaGraphLaunch(gexec[id], cs), "graph launch");
    note_launches((int)gkernels[id]);
  }

  // obj(v): one state solve. Results: dres[0] = sum (m(1) - m1)^2, dres[1] = regulariser sum.
  // With keep = true the state solve stores its trajectory (and v^, mu, X-) so that an immediately
  // following gradient(v) on the same, unmodified buffer reuses them instead of solving again.
  // w = alpha L v when the caller carries it (the solver), else nullptr (computed by the transform).
  void enqueue_objective(const T* v, const T* w, bool keep) {
    reg_dot(v, w, 1);
    if (needs_mu_forward() || keep) compute_mu(v);
    const T* mT;
    if (keep) {
      ck(launch_departure<T>(g, v, xm, xp, (T)ht, st, /*both=*/0), "departure");
      forward_all();
      mT = slot(nt);
    } else {
      mT = forward_final(v);
    }
    ck(launch_mismatch<T>(mT, m1, nullptr, nv, dpart, dres, st), "mismatch");
    issue_results(2);
  }
  double objective(const T* v, double* mismatch = nullptr, bool keep = false, const T* w = nullptr) {
    fwd_cache = nullptr;
    ck(cudaEventRecord(ev[0], st), "event");
    if (graphs && w && prof_class < 0) {
      ck(cudaMemcpyAsync(gin, v, sizeof(T) * vl, cudaMemcpyDeviceToDevice, st), "copy v");
      ck(cudaMemcpyAsync(gin + vl, w, sizeof(T) * vl, cudaMemcpyDeviceToDevice, st), "copy w");
      run_variant(keep ? G_OBJ_KEEP : G_OBJ, [&] { enqueue_objective(gin, gin + vl, keep); });
    } else {
      if (!w) {
        apply_alphaL(v, wtmp);
        w = wtmp;
      }
      enqueue_objective(v, w, keep);
    }
    ck(cudaEventRecord(ev[1], st), "event");
    wait_results();
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ev[0], ev[1]);
    ctx->stats.t_obj_ms += ms;
    ctx->stats.obj_evals += 1;
    ctx->stats.pde_solves += 1;
    const double m = 0.5 * hd * hres[0];
    if (mismatch) *mismatch = m;
    if (keep) fwd_cache = v;
    return m + reg_value(hres[1]);
  }
  const T* fwd_cache = nullptr;  // v whose trajectory, mu and X- are current (see objective)

  // Body force b (not projected) from the adjoint started at lam_init (lam_init may be lam[0]).
  // Requires departure points, mu and the forward states.
  // The trapezoid rule over t_j = j h_t, j = n_t .. 0, visits the time steps in pairs (j, j - 1): the
  // adjoint step to lambda_{j-1} is taken first, then one derivative pass per axis adds both steps'
  // terms (the two fields share each complex FFT). With n_t even, j = 0 is a single pass.
  // The derivative passes of a pair (a group) run on st2 once st has produced their operands, so they
  // overlap the next adjoint steps and segment recomputes on st; they still run one after another in
  // the same order, so b is summed exactly as on one stream. The adjoint states rotate through
  // kLamRing buffers and the recomputed segments through two: st overwrites a buffer only after the
  // group that read it is done. st waits for st2 at the end.
  // Precondition: the last forward_all ran on the same velocity (its last segment is in seg[0]; a
  // captured launch sequence therefore never depends on host state left by other calls).
  void body_force(const T* lam_init) {
    segs_after_forward();
    adjoint_chain_reset();
    ck(cudaMemsetAsync(body, 0, sizeof(T) * vl, st), "memset body");
    for (auto& r : lam_reader) r = -1;
    seg_reader[0] = seg_reader[1] = -1;
    bf_waited = -1;
    auto ring_of = [&](const T* p) {
      for (int i = 0; i < kLamRing; ++i)
        if (p == lam[i]) return i;
      return -1;
    };
    auto seg_of = [&](const T* p) {
      for (int b = 0; b < 2; ++b)
        if (seg[b] && p >= seg[b] && p < seg[b] + (long long)(K - 1) * nv) return b;
      return -1;
    };
    int ring = (ring_of(lam_init) + 1) % kLamRing;  // the next ring buffer to write
    auto next_lam = [&]() {
      const int i = ring;
      ring = (ring + 1) % kLamRing;
      bf_wait(lam_reader[i]);
      lam_reader[i] = -1;
      return lam[i];
    };
    int grp = 0;
    auto issue = [&](auto&& passes, const T* la, const T* lb, const T* ma, const T* mb) {
      ck(cudaEventRecord(bf_fork, st), "fork");
      ck(cudaStreamWaitEvent(st2, bf_fork, 0), "fork wait");
      passes();
      ck(cudaEventRecord(bf_ev[grp], st2), "group done");
      for (const T* p : {la, lb}) {
        const int i = p ? ring_of(p) : -1;
        if (i >= 0) lam_reader[i] = grp;
      }
      for (const T* p : {ma, mb}) {
        const int b = p ? seg_of(p) : -1;
        if (b >= 0) seg_reader[b] = grp;
      }
      ++grp;
    };
    const T* lcur = lam_init;
    const bool cont = model == GA_MODEL_CONTINUITY;
    auto coef_of = [&](int j) { return ht * ((j == 0 || j == nt) ? 0.5 : 1.0); };
    int j = nt;
    for (; j >= 1; j -= 2) {
      const T* mj = state(j);  // a stored state, or in the same segment as j - 1
      T* lprev = next_lam();
      sl_adjoint(lcur, lprev);  // lambda_{j-1}
      const T* mj1 = state(j - 1);
      const double c0 = coef_of(j), c1 = coef_of(j - 1);
      issue(
          [&] {
            for (int c = 0; c < dim; ++c) {
              if (cont)  // b -= h_t w_j pi_j grad lambda_j
                deriv_pair(g.axis_of(c), lcur, mj, -c0, lprev, mj1, -c1, body + c * nv, st2);
              else  // b += h_t w_j lambda_j grad m_j
                deriv_pair(g.axis_of(c), mj, lcur, c0, mj1, lprev, c1, body + c * nv, st2);
            }
          },
          lcur, lprev, mj, mj1);
      if (j - 1 >= 1) {
        T* lnext = next_lam();
        sl_adjoint(lprev, lnext);  // lambda_{j-2}
        lcur = lnext;
      } else {
        lcur = lprev;
      }
    }
    if (j == 0) {  // n_t even: the last time step alone
      const T* m0s = state(0);
      const double c0 = coef_of(0);
      issue(
          [&] {
            for (int c = 0; c < dim; ++c) {
              if (cont)
                deriv(g.axis_of(c), lcur, m0s, body + c * nv, -c0, true, st2);
              else
                deriv(g.axis_of(c), m0s, lcur, body + c * nv, c0, true, st2);
            }
          },
          lcur, nullptr, m0s, nullptr);
    }
    ck(cudaEventRecord(bf_join, st2), "join");
    ck(cudaStreamWaitEvent(st, bf_join, 0), "join wait");
    for (auto& r : lam_reader) r = -1;
    seg_reader[0] = seg_reader[1] = -1;
    bf_waited = -1;
  }

  // Reduced gradient g = alpha L v + (P) b (Eq. (3)) into gout (vl). w = alpha L v: carried by the
  // solver through every linear update of v, so the regulariser term never passes through a transform
  // of v whose rounding the symbol |k|^{2s} would amplify; nullptr computes it by the transform. When
  // s_out != nullptr, writes s = -(alpha L)^{-1} (P) g to s_out and alpha L s to s_out + vl.
  void enqueue_gradient(const T* v, const T* w, T* gout, T* s_out, bool reuse) {
    reg_dot(v, w, 1);
    if (reuse) {
      // mu, X- and the stored states are those of v: only X+ is missing
      ck(launch_departure<T>(g, v, xp, xm, (T)(-ht), st, /*both=*/0), "departure");
    } else {
      compute_mu(v);
      ck(launch_departure<T>(g, v, xm, xp, (T)ht, st), "departure");
      forward_all();
    }
    ck(launch_mismatch<T>(slot(nt), m1, lam[0], nv, dpart, dres, st), "mismatch");
    body_force(lam[0]);
    if (model == GA_MODEL_INCOMPRESSIBLE) {  // P b by the transform, in place
      for (int c = 0; c < dim; ++c) r2c(body + c * nv, bh + c * g.nhalf);
      SpecArgs sp{SPEC_LERAY, s, alpha, 1};
      ck(launch_spectral<T>(g, sp, bh, st), "spectral leray");
      for (int c = 0; c < dim; ++c) c2r(bh + c * g.nhalf, body + c * nv);
    }
    ck(launch_axpy<T>(gout, body, w, 1.0, vl, st), "g = (P) b + w");
    if (s_out) precond_into(gout, s_out, s_out + vl);
    ck(launch_maxabs<T>(gout, vl, dpart, dres + 2, st), "maxabs");
    issue_results(3);
  }
  double gradient(const T* v, T* gout, T* s_out, double* mismatch = nullptr, const T* w = nullptr) {
    ck(cudaEventRecord(ev[0], st), "event");
    const bool reuse = fwd_cache == v;  // trajectory of the last objective(v, .., keep) call
    fwd_cache = nullptr;
    if (graphs && w && prof_class < 0 && (!s_out || s_out == S)) {
      ck(cudaMemcpyAsync(gin, v, sizeof(T) * vl, cudaMemcpyDeviceToDevice, st), "copy v");
      ck(cudaMemcpyAsync(gin + vl, w, sizeof(T) * vl, cudaMemcpyDeviceToDevice, st), "copy w");
      const int id = s_out ? (reuse ? G_GRAD_REUSE_S : G_GRAD_S) : (reuse ? G_GRAD_REUSE : G_GRAD);
      run_variant(id, [&] { enqueue_gradient(gin, gin + vl, gbuf, s_out, reuse); });
      ck(cudaMemcpyAsync(gout, gbuf, sizeof(T) * vl, cudaMemcpyDeviceToDevice, st), "copy g");
    } else {
      if (!w) {
        apply_alphaL(v, wtmp);
        w = wtmp;
      }
      enqueue_gradient(v, w, gout, s_out, reuse);
    }
    ck(cudaEventRecord(ev[1], st), "event");
    wait_results();
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ev[0], ev[1]);
    ctx->stats.t_grad_ms += ms;
    ctx->stats.grad_evals += 1;
    ctx->stats.pde_solves += reuse ? 1 : 2;
    const double m = 0.5 * hd * hres[0];
    if (mismatch) *mismatch = m;
    const double val = m + reg_value(hres[1]);
    if (!std::isfinite(val) || !std::isfinite(hres[2])) {
      set_err(ctx, "non-finite objective or gradient (obj=%g, |g|inf=%g)", val, hres[2]);
      throw Fail{GA_ERR_NAN};
    }
    last_ginf = hres[2];
    return val;
  }
  double last_ginf = 0.0;

  void precond(const T* gin, T* sout) {
    precond_into(gin, sout, nullptr);
  }
  double dot_l2(const T* a, const T* b) {
    const T* bl[1] = {b};
    ck(launch_dots<T>(a, bl, 1, vl, dpart, dres + 8, st), "dots");
    read_results(9);
    return hd * hres[8];
  }

  // ---- deformation diagnostics ------------------------------------------------------------------
  // Displacement u (grid units, dim fields) of the map y = x + h u with m(., 1) = m0(y) and
  // det grad y, for a stationary velocity v. y composes the state step's departure points:
  // u_0 = 0, u_{j+1} = I[u_j](X-) + (X- - x). det grad y, the Jacobian of the inverse flow map, is
  // the density of the transported uniform measure: the continuity state solve from 1.
  void deformation(const T* v, T* u, T* detj) {
    compute_mu(v);
    ck(launch_departure<T>(g, v, xm, xp, (T)ht, st, 0), "departure");
    ck(cudaMemsetAsync(u, 0, sizeof(T) * vl, st), "memset");
    for (int c = 0; c < dim; ++c) {
      T* uc = u + c * nv;
      for (int j = 0; j < nt; ++j) {
        ck(launch_sl_forward<T>(g, 0, uc, xm, mu, tmp[0], (T)ht, st), "sl displacement");
        ck(launch_axpy<T>(uc, tmp[0], xm + c * nv, 1.0, nv, st), "displacement step");
      }
    }
    ck(launch_fill<T>(detj, 1.0, nv, st), "fill");
    T* a = detj;
    T* b = tmp[0];
    for (int j = 0; j < nt; ++j) {
      ck(launch_sl_forward<T>(g, 1, a, xm, mu, b, (T)ht, st), "sl det");
      std::swap(a, b);
    }
    if (a != detj) ck(cudaMemcpyAsync(detj, a, sizeof(T) * nv, cudaMemcpyDeviceToDevice, st), "copy det");
  }

  // ---- discretise-then-optimise gradient (advection transport; dto_kernels.cu) --------------------
  T* dto_buf = nullptr;  // Euclidean velocity gradient of the data term (allocated on first use)

  void dto_require_advection(const char* what) {
    if (model == GA_MODEL_CONTINUITY) {
      set_err(ctx, "%s: the discrete gradient is built for the advection transport (advection and "
                   "incompressible models)", what);
      throw Fail{GA_ERR_ARG};
    }
  }
  // Departure points and the forward states of v (stored or checkpointed).
  void dto_forward(const T* v) {
    ck(launch_departure<T>(g, v, xm, xp, (T)ht, st, /*both=*/0), "departure");
    forward_all();
  }
  // Euclidean gradient of coef <rT, m_{n_t}(v)> with respect to the grid values of v, into out:
  // r_{n_t} = rT, r_j = A^T r_{j+1}, G += coef r_{j+1} grad I[m_j](X-), then the chain rule through X-.
  void dto_backward(const T* v, const T* rT, double coef, T* out) {
    T* G = body;
    ck(cudaMemsetAsync(G, 0, sizeof(T) * vl, st), "memset G");
    if (rT != lam[0]) ck(cudaMemcpyAsync(lam[0], rT, sizeof(T) * nv, cudaMemcpyDeviceToDevice, st), "copy r");
    int pp = 0;
    segs_after_forward();  // dto_forward ran just before on the same v
    for (int j = nt - 1; j >= 0; --j) {
      const T* mj = state(j);
      ck(launch_dto_accum<T>(g, lam[pp], mj, xm, G, (T)coef, st), "dto accumulate");
      if (j > 0) {
        ck(cudaMemsetAsync(lam[pp ^ 1], 0, sizeof(T) * nv, st), "memset r");
        ck(launch_interp_scatter<T>(g, lam[pp], xm, lam[pp ^ 1], st), "interpolation transpose");
        pp ^= 1;
      }
    }
    ck(launch_dto_velocity<T>(g, v, G, out, (T)ht, st), "dto velocity");
  }
  // L2 gradient of the discrete objective: alpha L v + (P) (1/h^d) dJ_data/dv.
  double gradient_dto(const T* v, T* gout, double* mismatch) {
    dto_require_advection("ga_gradient_dto");
    if (!dto_buf) dto_buf = dalloc<T>(vl);
    fwd_cache = nullptr;
    ck(cudaEventRecord(ev[0], st), "event");
    apply_alphaL(v, wtmp);
    reg_dot(v, wtmp, 1);
    dto_forward(v);
    ck(launch_mismatch<T>(slot(nt), m1, lam[0], nv, dpart, dres, st), "mismatch");  // lam[0] = m1 - m(1)
    dto_backward(v, lam[0], -hd, dto_buf);  // r = h^d (m(1) - m1) = -h^d lam[0]
    if (model == GA_MODEL_INCOMPRESSIBLE) {
      for (int c = 0; c < dim; ++c) r2c(dto_buf + c * nv, bh + c * g.nhalf);
      SpecArgs sp{SPEC_LERAY, s, alpha, 1};
      ck(launch_spectral<T>(g, sp, bh, st), "spectral leray");
      for (int c = 0; c < dim; ++c) c2r(bh + c * g.nhalf, dto_buf + c * nv);
    }
    ck(launch_axpy<T>(gout, wtmp, dto_buf, 1.0 / hd, vl, st), "g = alpha L v + b / h^d");
    ck(launch_maxabs<T>(gout, vl, dpart, dres + 2, st), "maxabs");
    ck(cudaEventRecord(ev[1], st), "event");
    read_results(3);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ev[0], ev[1]);
    ctx->stats.t_grad_ms += ms;
    ctx->stats.grad_evals += 1;
    ctx->stats.pde_solves += 2;
    const double m = 0.5 * hd * hres[0];
    if (mismatch) *mismatch = m;
    const double val = m + reg_value(hres[1]);
    if (!std::isfinite(val) || !std::isfinite(hres[2])) {
      set_err(ctx, "non-finite objective or gradient (obj=%g, |g|inf=%g)", val, hres[2]);
      throw Fail{GA_ERR_NAN};
    }
    return val;
  }

  // ---- solver (Alg. 3) -----------------------------------------------------------------------------
  // ---- device-driven solve (ga_solver_opts.graphs == 2) ------------------------------------------
  // Fixed roles: the iterate v and w = alpha L v in VC with its gradient in GC; the line-search trial q
  // (and alpha L q) in Q with its gradient in GQ; the window in a ring of W1 slots (RV: v and w, RG: g)
  // indexed on the device (ResCtl). One graph holds a whole solve:
  //   IF (!started) { w = alpha L v; g, s at v; push }         (start of Alg. 3)
  //   WHILE (k < kmax, no failure, not converged) {
  //     <g, s>;  WHILE (trial rejected) { q = v + rho s; obj(q) keeping its trajectory; Armijo }
  //     SWITCH (step kind) { 0: g, s at q; v = q  |  1: g at q; window least squares; v = q + sum
  //       beta_i (q - v_i); g, s at v }
  //     push (v, g) into the window; k += 1; stop test }
  // and its kernels are the ones the host-driven solver launches, in the same order on the same data, so
  // both give the same iterates bit for bit.
  bool resident = false, rstarted = false;
  ResCtl* dctl = nullptr;
  ResCtl* hctl = nullptr;  // pinned copy of *dctl as of the last launch
  T *VC = nullptr, *GC = nullptr, *Q = nullptr, *GQ = nullptr, *RV = nullptr, *RG = nullptr;
  cudaStream_t cap[3] = {};  // capture streams, one per nesting level of the graph
  cudaGraphExec_t rexec = nullptr;
  // kernels recorded per body of the graph (for the launch count of a run)
  long long rk_fixed = 0, rk_start = 0, rk_iter = 0, rk_trial = 0, rk_fp = 0, rk_ga = 0;

  cudaGraph_t capturing_graph() {
    cudaStreamCaptureStatus cst;
    cudaGraph_t gr = nullptr;
    ck(cudaStreamGetCaptureInfo(st, &cst, nullptr, &gr, nullptr, nullptr, nullptr), "capture info");
    return gr;
  }
  cudaGraphConditionalHandle new_handle() {
    cudaGraphConditionalHandle h;
    ck(cudaGraphConditionalHandleCreate(&h, capturing_graph(), 0, 0), "conditional handle");
    return h;
  }
  // Appends a conditional node after the work captured so far on st; returns its body graphs.
  cudaGraph_t* add_conditional(cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type, unsigned size) {
    cudaStreamCaptureStatus cst;
    cudaGraph_t gr = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    ck(cudaStreamGetCaptureInfo(st, &cst, nullptr, &gr, &deps, nullptr, &nd), "capture info");
    cudaGraphNodeParams p{};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = h;
    p.conditional.type = type;
    p.conditional.size = size;
    cudaGraphNode_t node;
    ck(cudaGraphAddNode(&node, gr, deps, nullptr, nd, &p), "conditional node");
    ck(cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies),
       "capture dependencies");
    return p.conditional.phGraph_out;
  }
  // Records f() into graph `into` (a new chain with no dependencies) on capture stream `lvl`; returns
  // the number of kernels recorded.
  template <typename F> long long capture_to(cudaGraph_t into, int lvl, F&& f) {
    cudaStream_t cs = cap[lvl];
    const long long c0 = t_launches;
    ck(cudaStreamBeginCaptureToGraph(cs, into, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal),
       "begin capture");
    cudaStream_t saved = st;
    st = cs;
    try {
      f();
    } catch (...) {
      st = saved;
      cudaGraph_t gr = nullptr;
      cudaStreamEndCapture(cs, &gr);
      throw;
    }
    st = saved;
    cudaGraph_t gr = nullptr;
    ck(cudaStreamEndCapture(cs, &gr), "end capture");
    return t_launches - c0;
  }

  void res_push(int iteration, cudaGraphConditionalHandle h_iter) {
    ck(launch_ring_store<T>(RV, 2 * vl, dctl, W1, VC, 2 * vl, st), "ring v");
    ck(launch_ring_store<T>(RG, vl, dctl, W1, GC, vl, st), "ring g");
    ck(launch_dots_ring<T>(GC, GC, RG, vl, dctl, W1, 1, vl, dpart, dres + kResDots, st), "window dots");
    ck(launch_gram_push_ring(dM, W1, dctl, dres + kResDots, st), "gram push");
    ck(launch_res_pushed(dctl, iteration, h_iter, st), "window push");
  }

  // Adds this problem's whole solve to `top` as an independent chain of nodes.
  void add_resident(cudaGraph_t top) {
    const int saved_prof = prof_class;
    prof_class = -1;
    host_results = false;
    const long long c0 = t_launches;
    try {
      long long inner = 0;
      capture_to(top, 0, [&] {
        const cudaGraphConditionalHandle h_start = new_handle(), h_iter = new_handle();
        ck(launch_res_enter(dctl, h_start, st), "enter");
        cudaGraph_t* b = add_conditional(h_start, cudaGraphCondTypeIf, 1);
        rk_start = capture_to(b[0], 1, [&] {
          apply_alphaL(VC, VC + vl);
          enqueue_gradient(VC, VC + vl, GC, S, false);
          ck(launch_res_grad(dctl, dres, RES_GRAD_START, st), "start");
          res_push(0, 0);
        });
        ck(launch_res_loop_cond(dctl, h_iter, st), "loop condition");
        cudaGraph_t* l = add_conditional(h_iter, cudaGraphCondTypeWhile, 1);
        rk_iter = capture_to(l[0], 1, [&] {
          const T* bl[1] = {S};
          ck(launch_dots<T>(GC, bl, 1, vl, dpart, dres + 8, st), "<g, s>");
          const cudaGraphConditionalHandle h_ls = new_handle();
          ck(launch_res_ls_begin(dctl, dres + 8, h_ls, st), "line search");
          cudaGraph_t* lb = add_conditional(h_ls, cudaGraphCondTypeWhile, 1);
          rk_trial = capture_to(lb[0], 2, [&] {
            ck(launch_axpy_dev<T>(Q, VC, S, &dctl->rho, 2 * vl, st), "q = v + rho s");
            enqueue_objective(Q, Q + vl, true);
            ck(launch_res_ls_check(dctl, dres, h_ls, st), "Armijo test");
          });
          const cudaGraphConditionalHandle h_sw = new_handle();
          ck(launch_res_branch(dctl, h_sw, st), "step kind");
          cudaGraph_t* sw = add_conditional(h_sw, cudaGraphCondTypeSwitch, 2);
          rk_fp = capture_to(sw[0], 2, [&] {  // fixed-point step: v <- q
            enqueue_gradient(Q, Q + vl, GQ, S, true);
            ck(launch_res_grad(dctl, dres, RES_GRAD_ACCEPTED, st), "gradient");
            ck(cudaMemcpyAsync(VC, Q, sizeof(T) * 2 * vl, cudaMemcpyDeviceToDevice, st), "copy q");
            ck(cudaMemcpyAsync(GC, GQ, sizeof(T) * vl, cudaMemcpyDeviceToDevice, st), "copy g");
          });
          rk_ga = capture_to(sw[1], 2, [&] {  // NGMRES step: v <- q + sum_i beta_i (q - v_i)
            enqueue_gradient(Q, Q + vl, GQ, nullptr, true);
            ck(launch_res_grad(dctl, dres, RES_GRAD_TRIAL, st), "gradient");
            ck(launch_dots_ring<T>(GQ, GQ, RG, vl, dctl, W1, 0, vl, dpart, dres + kResDots, st), "lsq dots");
            ck(launch_lsq_ring(dctl, W1, dres + kResDots, dM, dbeta, dres + kResLsq, st), "lsq");
            ck(launch_combine_ring<T>(VC, Q, RV, 2 * vl, dctl, W1, dbeta, 2 * vl, st), "combine");
            enqueue_gradient(VC, VC + vl, GC, S, false);
            ck(launch_res_grad(dctl, dres, RES_GRAD_COMBINED, st), "gradient");
          });
          res_push(1, h_iter);
        });
        inner = rk_start + rk_iter;
      });
      rk_iter -= rk_trial + rk_fp + rk_ga;  // kernels of an iteration outside its nested bodies
      rk_fixed = (t_launches - c0) - inner;  // enter and loop condition
    } catch (...) {
      host_results = true;
      prof_class = saved_prof;
      note_launches((int)-(t_launches - c0));
      throw;
    }
    host_results = true;
    prof_class = saved_prof;
    note_launches((int)-(t_launches - c0));  // recorded, not launched
  }

  // Host side of a run: parameters into the pinned copy (a fresh run also clears the state, so the
  // graph starts the solve from VC), then copied to the device on st.
  void res_prepare(bool fresh, int kmax, int stop) {
    if (fresh) std::memset(hctl, 0, sizeof(ResCtl));
    const ga_solver_opts& o = ctx->opts;
    hctl->armijo_c = o.armijo_c;
    hctl->rel_tol = o.rel_tol;
    hctl->hd = hd;
    hctl->max_backtracks = o.max_backtracks;
    hctl->sigma = o.sigma;
    hctl->tau = o.tau;
    hctl->variant = o.variant;
    hctl->method = o.method;
    hctl->W1 = W1;
    hctl->kmax = kmax;
    hctl->stop_on_converged = stop;
    res_before = *hctl;
    ck(cudaMemcpyAsync(dctl, hctl, sizeof(ResCtl), cudaMemcpyHostToDevice, st), "control upload");
  }
  ResCtl res_before{};
  void res_fetch() { ck(cudaMemcpyAsync(hctl, dctl, sizeof(ResCtl), cudaMemcpyDeviceToHost, st), "control download"); }
  // After the stream has synchronised: statistics, launch count and status of the run.
  // `ms`: device time of the run (evaluations and control are not timed apart; added to t_grad_ms).
  void res_finish(float ms) {
    const ResCtl& c = *hctl;
    const ResCtl& b = res_before;
    const long long iters = c.k - b.k, trials = c.ls_trials - b.ls_trials, fps = c.fp_steps - b.fp_steps;
    long long n = rk_fixed + (b.started ? 0 : rk_start) + iters * rk_iter + trials * rk_trial + fps * rk_fp +
                  (iters - fps) * rk_ga;
    if (c.status != 0 && c.started) {  // the failed iteration ran its kernels but did not count itself
      n += rk_iter;
      if (c.branch == 0) n += rk_fp;
      if (c.branch == 1) n += rk_ga;
    }
    note_launches((int)n);
    ga_stats& o = ctx->stats;
    if (!b.started) o = ga_stats{};
    o.t_grad_ms += ms;
    o.iters = c.k;
    o.grad_evals = (int)c.grad_evals;
    o.obj_evals = (int)c.obj_evals;
    o.pde_solves = (int)c.pde_solves;
    o.ls_trials = (int)c.ls_trials;
    o.last_branch = c.last_branch;
    o.converged = c.converged;
    o.obj = c.J;
    o.mismatch = c.mis;
    o.rel_grad_inf = c.rel_grad_inf;
    o.grad_inf0 = c.g0inf;
    o.rho_mem = c.rho_mem;
    o.last_rho = c.last_rho;
    k = c.k;
    if (c.status != 0) {
      rstarted = false;
      if (c.status == kResErrLinesearch)
        set_err(ctx, "Armijo line search failed after %d halvings (iteration %d)", ctx->opts.max_backtracks, c.k);
      else
        set_err(ctx, "non-finite objective or gradient (iteration %d)", c.k);
      throw Fail{(ga_status)c.status};
    }
    rstarted = true;
  }
  void res_build() {
    if (rexec) return;
    cudaGraph_t top = nullptr;
    ck(cudaGraphCreate(&top, 0), "graph create");
    try {
      add_resident(top);
    } catch (...) {
      cudaGraphDestroy(top);
      throw;
    }
    const cudaError_t e = cudaGraphInstantiate(&rexec, top, 0);
    cudaGraphDestroy(top);
    ck(e, "graph instantiate");
  }
  // Runs the solve's graph on st until k = kmax (or convergence when stop != 0). A fresh run starts from
  // vin (device, vl values); otherwise it continues from the state of the last run.
  void res_run(const T* vin, bool fresh, int kmax, int stop) {
    res_build();
    res_stage(vin, fresh, kmax, stop);
    ck(cudaEventRecord(ev[0], st), "event");
    ck(cudaGraphLaunch(rexec, st), "graph launch");
    ck(cudaEventRecord(ev[1], st), "event");
    res_complete();
  }
  void res_stage(const T* vin, bool fresh, int kmax, int stop) {
    if (fresh) ck(cudaMemcpyAsync(VC, vin, sizeof(T) * vl, cudaMemcpyDeviceToDevice, st), "copy v");
    res_prepare(fresh, kmax, stop);
  }
  // After the run's launch on st (bracketed by ev[0] and ev[1]): fetch the control block and finish.
  void res_complete() {
    res_fetch();
    ck(cudaStreamSynchronize(st), "sync");
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ev[0], ev[1]);
    res_finish(ms);
  }

  void reset() {
    while (!win.empty()) {
      vfree.push_back(win.back().first);
      gfree.push_back(win.back().second);
      win.pop_back();
    }
    while (!awin.empty()) {
      vfree.push_back(awin.back().first);
      gfree.push_back(awin.back().second);
      awin.pop_back();
    }
    if (cur_v) vfree.push_back(cur_v);
    if (cur_g) gfree.push_back(cur_g);
    cur_v = cur_g = nullptr;
    started = false;
    s_valid = false;
    k = 0;
    rho_mem = 1.0;
    g0inf = 0.0;
    ctx->stats = ga_stats{};
    ctx->stats.rho_mem = 1.0;
    rstarted = false;
  }

  T* take(std::vector<T*>& pool) {
    T* p = pool.back();
    pool.pop_back();
    return p;
  }

  // Append (v, g) as the newest window entry; update the device Gram of the window gradients.
  void push_window(T* v, T* gv) {
    int keep = (int)win.size();
    if (keep == W1) {
      vfree.push_back(win.back().first);
      gfree.push_back(win.back().second);
      win.pop_back();
      keep = W1 - 1;
    }
    std::vector<const T*> bl;
    bl.push_back(gv);
    for (int i = 0; i < keep; ++i) bl.push_back(win[i].second);
    ck(launch_dots<T>(gv, bl.data(), (int)bl.size(), vl, dpart, dres + kResDots, st), "window dots");
    ck(launch_gram_push(dM, W1, keep, dres + kResDots, st), "gram push");
    win.push_front({v, gv});
  }

  // GA-AA state: the current iterate and its gradient, and the previous (q_j, r_j = v_j - q_j),
  // newest first, at most w entries; dM then holds the Gram matrix of the window residuals.
  std::deque<std::pair<T*, T*>> awin;
  T* cur_v = nullptr;
  T* cur_g = nullptr;

  bool aa() const { return ctx->opts.method == GA_METHOD_GA_AA; }
  T* current() const { return resident ? VC : (aa() ? cur_v : win.front().first); }

  // Append (q, r) as the newest GA-AA window entry, dropping the oldest beyond w entries.
  void push_aa(T* q, T* r) {
    if (W1 == 1) {  // w = 0: nothing is kept
      vfree.push_back(q);
      gfree.push_back(r);
      return;
    }
    int keep = (int)awin.size();
    if (keep == W1 - 1) {
      vfree.push_back(awin.back().first);
      gfree.push_back(awin.back().second);
      awin.pop_back();
      keep = W1 - 2;
    }
    std::vector<const T*> bl;
    bl.push_back(r);
    for (int i = 0; i < keep; ++i) bl.push_back(awin[i].second);
    ck(launch_dots<T>(r, bl.data(), (int)bl.size(), vl, dpart, dres + kResDots, st), "window dots");
    ck(launch_gram_push(dM, W1, keep, dres + kResDots, st), "gram push");
    awin.push_front({q, r});
  }

  bool is_fp_step(int kk) const {
    const ga_solver_opts& o = ctx->opts;
    if (o.method == GA_METHOD_RPGD) return true;
    const int per = o.sigma + o.tau;
    return o.variant == 2 ? (kk % per) < o.tau : (kk % per) >= o.sigma;
  }

  void start(const T* v0) {
    reset();
    T* v = take(vfree);
    T* gv = take(gfree);
    ck(cudaMemcpyAsync(v, v0, sizeof(T) * vl, cudaMemcpyDeviceToDevice, st), "copy v0");
    apply_alphaL(v, v + vl);  // from here on w = alpha L v follows every linear update of v
    J = gradient(v, gv, S, &mis, v + vl);
    s_valid = true;
    g0inf = last_ginf;
    if (aa()) {
      cur_v = v;
      cur_g = gv;
    } else {
      push_window(v, gv);
    }
    started = true;
    ga_stats& stt = ctx->stats;
    stt.obj = J;
    stt.mismatch = mis;
    stt.grad_inf0 = g0inf;
    stt.rel_grad_inf = g0inf > 0 ? 1.0 : 0.0;
    stt.rho_mem = rho_mem;
  }

  // q(v) = v + rho s by the Armijo line search with step memory (Eqs. (6)-(7), Sec. 2.3), s = S the
  // preconditioned direction at v. Returns the accepted trial in a buffer of the v pool; its state
  // trajectory stays cached for a gradient evaluation at exactly that buffer.
  T* qmap(const T* v, const T* gv) {
    const ga_solver_opts& o = ctx->opts;
    ga_stats& stt = ctx->stats;
    if (!s_valid) precond_into(gv, S, S + vl);
    const double gs = dot_l2(gv, S);
    T* q = take(vfree);
    double rho = rho_mem, Jq = 0.0;
    bool ok = false;
    for (int it = 0; it <= o.max_backtracks; ++it) {
      ck(launch_axpy<T>(q, v, S, rho, 2 * vl, st), "axpy");  // q = v + rho s and alpha L q
      Jq = objective(q, nullptr, /*keep=*/true, q + vl);
      stt.ls_trials += 1;
      if (Jq < J + o.armijo_c * rho * gs) {
        rho_mem = (it == 0) ? 2.0 * rho : rho;
        ok = true;
        break;
      }
      rho *= 0.5;
    }
    if (!ok) {
      vfree.push_back(q);
      set_err(ctx, "Armijo line search failed after %d halvings (iteration %d)", o.max_backtracks, k);
      throw Fail{GA_ERR_LINESEARCH};
    }
    stt.last_rho = rho;
    stt.rho_mem = rho_mem;
    return q;
  }

  void finish_step(bool fp, double Jn, double misn) {
    const ga_solver_opts& o = ctx->opts;
    ga_stats& stt = ctx->stats;
    s_valid = true;
    J = Jn;
    ++k;
    stt.iters = k;
    stt.last_branch = fp ? 1 : 0;
    stt.obj = Jn;
    stt.mismatch = misn;
    stt.rel_grad_inf = g0inf > 0 ? last_ginf / g0inf : 0.0;
    stt.converged = stt.rel_grad_inf <= o.rel_tol ? 1 : 0;
  }

  // One iteration k of GA-AA(w; sigma, tau): Anderson acceleration AA(w) (Alg. 2) on the fixed-point
  // map q with the mixing schedule of Alg. 3. With r_j = v_j - q(v_j), the coefficients xi minimise
  // ||r_k + sum_{i=1..w^(k)} xi_i (r_k - r_{k-i})|| and v_{k+1} = q_k + sum_i xi_i (q_k - q_{k-i});
  // a fixed-point step (or an empty window) takes v_{k+1} = q_k. Both kinds of step enter the window.
  void step_aa() {
    T* v = cur_v;
    T* gv = cur_g;
    T* q = qmap(v, gv);
    T* r = take(gfree);
    ck(launch_axpy<T>(r, v, q, -1.0, vl, st), "residual");
    const bool fp = is_fp_step(k) || awin.empty();
    T *vn, *gn = take(gfree);
    double Jn, misn;
    if (fp) {
      Jn = gradient(q, gn, S, &misn, q + vl);  // reuses the accepted trial's state trajectory
      vn = q;
      if (W1 > 1) {
        T* qw = take(vfree);
        ck(cudaMemcpyAsync(qw, q, sizeof(T) * 2 * vl, cudaMemcpyDeviceToDevice, st), "copy q");
        push_aa(qw, r);
      } else {
        gfree.push_back(r);
      }
    } else {
      const int m = (int)awin.size();  // w^(k) previous entries
      std::vector<const T*> bl;
      bl.push_back(r);
      for (int i = 0; i < m; ++i) bl.push_back(awin[i].second);
      ck(launch_dots<T>(r, bl.data(), (int)bl.size(), vl, dpart, dres + kResDots, st), "lsq dots");
      ck(launch_lsq(m, dres + kResDots, dM, W1, dbeta, dres + kResLsq, st), "lsq");
      vn = take(vfree);
      std::vector<const T*> qlst;
      for (int i = 0; i < m; ++i) qlst.push_back(awin[i].first);
      ck(launch_combine<T>(vn, q, qlst.data(), dbeta, m, 2 * vl, st), "combine");  // v and alpha L v
      push_aa(q, r);  // stream order keeps a dropped entry intact until the combination has read it
      Jn = gradient(vn, gn, S, &misn, vn + vl);
    }
    vfree.push_back(cur_v);
    gfree.push_back(cur_g);
    cur_v = vn;
    cur_g = gn;
    finish_step(fp, Jn, misn);
  }

  // One iteration k of Alg. 3 (or of RPGD, or of GA-AA). For GA-NGMRES and RPGD the current iterate
  // is the newest window entry.
  void step() {
    if (aa()) {
      step_aa();
      return;
    }
    T* v = win.front().first;
    T* gv = win.front().second;
    T* q = qmap(v, gv);
    const bool fp = is_fp_step(k);
    T* gq = take(gfree);
    T *vn, *gn;
    double Jn, misn;
    if (fp) {
      Jn = gradient(q, gq, S, &misn, q + vl);
      vn = q;
      gn = gq;
    } else {
      double misq;
      gradient(q, gq, nullptr, &misq, q + vl);
      const int m = (int)win.size();  // w^(k) + 1 window entries
      std::vector<const T*> bl;
      bl.push_back(gq);
      for (int i = 0; i < m; ++i) bl.push_back(win[i].second);
      ck(launch_dots<T>(gq, bl.data(), (int)bl.size(), vl, dpart, dres + kResDots, st), "lsq dots");
      ck(launch_lsq(m, dres + kResDots, dM, W1, dbeta, dres + kResLsq, st), "lsq");
      vn = take(vfree);
      std::vector<const T*> vlst;
      for (int i = 0; i < m; ++i) vlst.push_back(win[i].first);
      ck(launch_combine<T>(vn, q, vlst.data(), dbeta, m, 2 * vl, st), "combine");  // v and alpha L v
      vfree.push_back(q);
      gfree.push_back(gq);
      gn = take(gfree);
      Jn = gradient(vn, gn, S, &misn, vn + vl);
    }
    push_window(vn, gn);
    finish_step(fp, Jn, misn);
  }
};

// ================================================================================================
// C ABI
// ================================================================================================

namespace {

bool good_len(int n) {
  if (n < 4 || n > 1024) return false;
  FftPlan p;
  return make_plan(n, &p);
}

template <typename F> ga_status guard(ga_ctx* c, F&& f) {
  try {
    f();
    return GA_OK;
  } catch (const Fail& e) {
    return e.st;
  } catch (...) {
    set_err(c, "unexpected host exception");
    return GA_ERR_CUDA;
  }
}


// Run fn(engine) with the engine of the context's precision.
template <typename F> ga_status dispatch(ga_ctx* c, F&& fn) {
  if (!c) return GA_ERR_ARG;
  return guard(c, [&] {
    // the reuse of a line-search state solve never spans two calls of the C ABI
    if (c->ef) {
      c->ef->fwd_cache = nullptr;
      fn(*c->ef);
    } else {
      c->ed->fwd_cache = nullptr;
      fn(*c->ed);
    }
  });
}

// Copy a caller buffer of `count` elements into device staging (or use it directly).
template <typename T> const T* stage_in(Engine<T>& e, const void* p, long long count, int mem, T* staging) {
  if (mem == GA_MEM_DEVICE) return static_cast<const T*>(p);
  e.ck(cudaMemcpyAsync(staging, p, sizeof(T) * count, cudaMemcpyHostToDevice, e.st), "H2D copy");
  return staging;
}
template <typename T> void stage_out(Engine<T>& e, void* p, const T* src, long long count, int mem) {
  if (mem == GA_MEM_DEVICE) {
    if (p != static_cast<const void*>(src)) e.ck(cudaMemcpyAsync(p, src, sizeof(T) * count, cudaMemcpyDeviceToDevice, e.st), "D2D copy");
  } else {
    e.ck(cudaMemcpyAsync(p, src, sizeof(T) * count, cudaMemcpyDeviceToHost, e.st), "D2H copy");
  }
  e.ck(cudaStreamSynchronize(e.st), "sync");
}

}  // namespace

// One-launch batch graphs of the device-driven solve, by the exact list of contexts (dropped with any
// of them).
struct BatchGraph {
  std::vector<ga_ctx*> key;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  void release() {
    if (exec) cudaGraphExecDestroy(exec);
    if (stream) cudaStreamDestroy(stream);
    if (done) cudaEventDestroy(done);
    exec = nullptr;
    stream = nullptr;
    done = nullptr;
  }
};
static std::mutex g_batch_mu;
static std::deque<BatchGraph> g_batches;
static void drop_batches_of(ga_ctx* c) {
  std::lock_guard<std::mutex> lk(g_batch_mu);
  for (auto it = g_batches.begin(); it != g_batches.end();) {
    if (std::find(it->key.begin(), it->key.end(), c) != it->key.end()) {
      if (it->stream) cudaStreamSynchronize(it->stream);
      it->release();
      it = g_batches.erase(it);
    } else {
      ++it;
    }
  }
}

static thread_local std::string g_setup_err;

namespace ga {
void set_global_error(const char* msg) { g_setup_err = msg ? msg : ""; }
}  // namespace ga

static bool valid_setup(const ga_problem_desc& d, const ga_solver_opts& o) {
  bool ok = (d.dim == 2 || d.dim == 3) && d.nt >= 1 && d.nt <= 4096 && d.model >= 0 && d.model <= 2 &&
            d.reg_order >= 1 && d.reg_order <= 3 && d.alpha > 0.0 && std::isfinite(d.alpha) &&
            (d.prec == GA_PREC_FP64 || d.prec == GA_PREC_MIXED) && d.ckpt_every >= 0;
  for (int a = 0; ok && a < d.dim; ++a) ok = good_len(d.n[a]);
  return ok && o.window >= 0 && o.window < kMaxWin && o.window + 2 <= kMaxDots && o.sigma >= 1 && o.tau >= 0 &&
         o.max_iter >= 1 && o.rel_tol >= 0.0 && o.armijo_c > 0.0 && o.max_backtracks >= 0 &&
         o.max_backtracks <= 200 && (o.variant == 1 || o.variant == 2) &&
         (o.method == GA_METHOD_GA_NGMRES || o.method == GA_METHOD_RPGD || o.method == GA_METHOD_GA_AA) &&
         (o.graphs == 0 || o.graphs == 1 || (o.graphs == 2 && o.method != GA_METHOD_GA_AA));
}

// Bytes of the buffers ga_setup allocates on the device, from the same layout the engine allocates.
template <typename T> static size_t planned_bytes(const ga_problem_desc& d, const ga_solver_opts& o) {
  auto e = std::make_unique<Engine<T>>();
  e->derive(d, o);
  size_t b = 0;
  e->layout([&](auto*& p, long long count) {
    using U = std::remove_reference_t<decltype(*p)>;
    b += sizeof(U) * (size_t)std::max(count, 1LL);
  });
  return b;
}

static size_t planned_bytes(const ga_problem_desc& d, const ga_solver_opts& o) {
  return d.prec == GA_PREC_MIXED ? planned_bytes<float>(d, o) : planned_bytes<double>(d, o);
}

extern "C" {

const char* ga_status_str(ga_status s) {
  switch (s) {
    case GA_OK: return "GA_OK";
    case GA_ERR_ARG: return "GA_ERR_ARG";
    case GA_ERR_CUDA: return "GA_ERR_CUDA";
    case GA_ERR_NOMEM: return "GA_ERR_NOMEM";
    case GA_ERR_NAN: return "GA_ERR_NAN";
    case GA_ERR_LINESEARCH: return "GA_ERR_LINESEARCH";
    case GA_ERR_NOT_CONVERGED: return "GA_ERR_NOT_CONVERGED";
    case GA_ERR_TIMEOUT: return "GA_ERR_TIMEOUT";
  }
  return "GA_ERR_UNKNOWN";
}


const char* ga_last_error(const ga_ctx* ctx) {
  if (ctx) return ctx->err.c_str();
  return g_setup_err.empty() ? "null context" : g_setup_err.c_str();
}

ga_status ga_workspace_bytes(const ga_problem_desc* desc, const ga_solver_opts* opts, size_t* bytes) {
  if (!desc || !opts || !bytes) return GA_ERR_ARG;
  if (!valid_setup(*desc, *opts)) {
    g_setup_err = "invalid problem descriptor or solver options";
    return GA_ERR_ARG;
  }
  *bytes = planned_bytes(*desc, *opts);
  return GA_OK;
}

ga_status ga_setup(const ga_problem_desc* desc, const ga_solver_opts* opts, const void* m0, const void* m1,
                   int mem, void* stream, ga_ctx** out) {
  if (!out) return GA_ERR_ARG;
  *out = nullptr;
  if (!desc || !opts || !m0 || !m1) return GA_ERR_ARG;
  const ga_problem_desc& d = *desc;
  const ga_solver_opts& o = *opts;
  if (!valid_setup(d, o) || (mem != GA_MEM_HOST && mem != GA_MEM_DEVICE)) {
    g_setup_err = "invalid problem descriptor or solver options";
    return GA_ERR_ARG;
  }
  {  // refuse, before allocating anything, a workspace larger than the device's free memory
    const size_t need = planned_bytes(d, o);
    size_t free_b = 0, total_b = 0;
    const cudaError_t e = cudaMemGetInfo(&free_b, &total_b);
    if (e != cudaSuccess) {
      cudaGetLastError();
      g_setup_err = std::string("cudaMemGetInfo: ") + cudaGetErrorString(e);
      return GA_ERR_CUDA;
    }
    if (need > free_b) {
      char buf[192];
      std::snprintf(buf, sizeof buf, "the problem needs %zu bytes of device memory, %zu are free (of %zu)", need,
                    free_b, total_b);
      g_setup_err = buf;
      return GA_ERR_NOMEM;
    }
  }
  ga_ctx* c = new ga_ctx();
  c->desc = d;
  c->opts = o;
  c->st = static_cast<cudaStream_t>(stream);
  c->prec = d.prec;
  c->stats = ga_stats{};
  c->stats.rho_mem = 1.0;
  ga_status s = guard(c, [&] {
    if (d.prec == GA_PREC_MIXED) {
      c->ef = new Engine<float>();
      c->ef->init(c, m0, m1, mem);
    } else {
      c->ed = new Engine<double>();
      c->ed->init(c, m0, m1, mem);
    }
  });
  if (s != GA_OK) {
    g_setup_err = c->err;
    delete c->ef;
    delete c->ed;
    delete c;
    return s;
  }
  *out = c;
  return GA_OK;
}

void ga_destroy(ga_ctx* ctx) {
  if (!ctx) return;
  if (ctx->st) cudaStreamSynchronize(ctx->st);
  else cudaDeviceSynchronize();
  drop_batches_of(ctx);
  delete ctx->ef;
  delete ctx->ed;
  delete ctx;
}

ga_status ga_objective(ga_ctx* ctx, const void* v, int mem, double* obj) {
  if (!ctx || !v || !obj || (mem != GA_MEM_HOST && mem != GA_MEM_DEVICE)) return GA_ERR_ARG;
  return dispatch(ctx, [&](auto& e) {
    auto* vin = stage_in(e, v, e.vl, mem, e.io_a);
    const double J = e.objective(vin);
    if (!std::isfinite(J)) {
      set_err(ctx, "non-finite objective");
      throw Fail{GA_ERR_NAN};
    }
    *obj = J;
  });
}

ga_status ga_gradient(ga_ctx* ctx, const void* v, void* g, int mem, double* obj) {
  if (!ctx || !v || !g || (mem != GA_MEM_HOST && mem != GA_MEM_DEVICE)) return GA_ERR_ARG;
  return dispatch(ctx, [&](auto& e) {
    using T = typename std::remove_reference<decltype(*e.m0)>::type;
    auto* vin = stage_in(e, v, e.vl, mem, e.io_a);
    T* gout = mem == GA_MEM_DEVICE ? static_cast<T*>(g) : e.io_b;
    const double J = e.gradient(vin, gout, nullptr);
    if (obj) *obj = J;
    stage_out(e, g, gout, e.vl, mem);
  });
}

ga_status ga_deformation(ga_ctx* ctx, const void* v, void* u, void* detj, int mem) {
  if (!ctx || !v || !u || !detj || (mem != GA_MEM_HOST && mem != GA_MEM_DEVICE)) return GA_ERR_ARG;
  return dispatch(ctx, [&](auto& e) {
    using T = typename std::remove_reference<decltype(*e.m0)>::type;
    auto* vin = stage_in(e, v, e.vl, mem, e.io_a);
    T* uout = mem == GA_MEM_DEVICE ? static_cast<T*>(u) : e.io_b;
    T* jout = mem == GA_MEM_DEVICE ? static_cast<T*>(detj) : e.tmp[1];
    e.deformation(vin, uout, jout);
    stage_out(e, u, uout, e.vl, mem);
    stage_out(e, detj, jout, e.nv, mem);
  });
}

ga_status ga_gradient_dto(ga_ctx* ctx, const void* v, void* g, int mem, double* obj) {
  if (!ctx || !v || !g || (mem != GA_MEM_HOST && mem != GA_MEM_DEVICE)) return GA_ERR_ARG;
  return dispatch(ctx, [&](auto& e) {
    using T = typename std::remove_reference<decltype(*e.m0)>::type;
    auto* vin = stage_in(e, v, e.vl, mem, e.io_a);
    T* gout = mem == GA_MEM_DEVICE ? static_cast<T*>(g) : e.io_b;
    const double J = e.gradient_dto(vin, gout, nullptr);
    if (obj) *obj = J;
    stage_out(e, g, gout, e.vl, mem);
  });
}

ga_status ga_precond(ga_ctx* ctx, const void* g, void* s, int mem) {
  if (!ctx || !g || !s || (mem != GA_MEM_HOST && mem != GA_MEM_DEVICE)) return GA_ERR_ARG;
  return dispatch(ctx, [&](auto& e) {
    using T = typename std::remove_reference<decltype(*e.m0)>::type;
    auto* gin = stage_in(e, g, e.vl, mem, e.io_a);
    T* sout = mem == GA_MEM_DEVICE ? static_cast<T*>(s) : e.io_b;
    e.precond(gin, sout);
    stage_out(e, s, sout, e.vl, mem);
  });
}

ga_status ga_reset(ga_ctx* ctx) {
  if (!ctx) return GA_ERR_ARG;
  return dispatch(ctx, [&](auto& e) { e.reset(); });
}

ga_status ga_get_stats(const ga_ctx* ctx, ga_stats* stats) {
  if (!ctx || !stats) return GA_ERR_ARG;
  *stats = ctx->stats;
  return GA_OK;
}

ga_status ga_step(ga_ctx* ctx, void* v_inout, int mem, ga_stats* stats) {
  if (!ctx || !v_inout || (mem != GA_MEM_HOST && mem != GA_MEM_DEVICE)) return GA_ERR_ARG;
  const auto t0 = std::chrono::steady_clock::now();
  ga_status s = dispatch(ctx, [&](auto& e) {
    if (e.resident) {  // one iteration of the device-driven solve (a fresh start first if needed)
      const bool fresh = !e.rstarted;
      auto* vin = fresh ? stage_in(e, v_inout, e.vl, mem, e.io_a) : nullptr;
      e.res_run(vin, fresh, fresh ? 1 : e.k + 1, 0);
    } else {
      if (!e.started) {
        auto* vin = stage_in(e, v_inout, e.vl, mem, e.io_a);
        e.start(vin);
      }
      e.step();
    }
    stage_out(e, v_inout, e.current(), e.vl, mem);
  });
  ctx->stats.t_total_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (stats) *stats = ctx->stats;
  return s;
}

ga_status ga_solve(ga_ctx* ctx, void* v_inout, int mem, ga_stats* stats) {
  if (!ctx || !v_inout || (mem != GA_MEM_HOST && mem != GA_MEM_DEVICE)) return GA_ERR_ARG;
  const auto t0 = std::chrono::steady_clock::now();
  ga_status s = dispatch(ctx, [&](auto& e) {
    auto* vin = stage_in(e, v_inout, e.vl, mem, e.io_a);
    if (e.resident) {  // the whole solve is one graph launch
      e.res_run(vin, true, ctx->opts.max_iter, 1);
      stage_out(e, v_inout, e.current(), e.vl, mem);
      return;
    }
    e.start(vin);
    if (ctx->stats.rel_grad_inf > ctx->opts.rel_tol) {
      while (e.k < ctx->opts.max_iter) {
        e.step();
        if (ctx->stats.converged) break;
      }
    } else {
      ctx->stats.converged = 1;
    }
    stage_out(e, v_inout, e.current(), e.vl, mem);
  });
  ctx->stats.t_total_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (stats) *stats = ctx->stats;
  if (s == GA_OK && !ctx->stats.converged) return GA_ERR_NOT_CONVERGED;
  return s;
}

// The status of a batch: the first failure in problem order, else GA_ERR_NOT_CONVERGED if any problem
// hit its iteration cap, else GA_OK.
static ga_status batch_status(int count, ga_ctx* const* ctxs, const std::vector<ga_status>& st) {
  ga_status worst = GA_OK;
  for (int i = 0; i < count; ++i) {
    if (st[i] == GA_ERR_NOT_CONVERGED) {
      if (worst == GA_OK) worst = st[i];
    } else if (st[i] != GA_OK) {
      ga::set_global_error(("problem " + std::to_string(i) + ": " + ctxs[i]->err).c_str());
      return st[i];
    }
  }
  return worst;
}

// All contexts device-driven: every problem's whole solve is one chain of the same graph, launched
// once; the graph is kept for the next call with the same contexts.
static ga_status solve_batch_resident(int count, ga_ctx* const* ctxs, void* const* v, int mem, ga_stats* stats) {
  std::lock_guard<std::mutex> lk(g_batch_mu);
  std::vector<ga_status> st(count, GA_OK);
  for (int i = 0; i < count; ++i) {
    ga_ctx* c = ctxs[i];
    const ga_status s = dispatch(c, [&](auto& e) {
      auto* vin = stage_in(e, v[i], e.vl, mem, e.io_a);
      e.res_stage(vin, true, c->opts.max_iter, 1);
      e.ck(cudaEventRecord(e.ev[0], e.st), "event");
    });
    if (s != GA_OK) {
      ga::set_global_error(("problem " + std::to_string(i) + ": " + c->err).c_str());
      return s;
    }
  }
  const std::vector<ga_ctx*> key(ctxs, ctxs + count);
  BatchGraph* bg = nullptr;
  for (auto& b : g_batches)
    if (b.key == key) bg = &b;
  if (!bg) {
    BatchGraph nb;
    nb.key = key;
    cudaGraph_t top = nullptr;
    cudaError_t e = cudaGraphCreate(&top, 0);
    for (int i = 0; i < count && e == cudaSuccess; ++i) {
      const ga_status s = dispatch(ctxs[i], [&](auto& en) { en.add_resident(top); });
      if (s != GA_OK) {
        cudaGraphDestroy(top);
        ga::set_global_error(("problem " + std::to_string(i) + ": " + ctxs[i]->err).c_str());
        return s;
      }
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&nb.exec, top, 0);
    if (top) cudaGraphDestroy(top);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&nb.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&nb.done, cudaEventDisableTiming);
    if (e != cudaSuccess) {
      nb.release();
      ga::set_global_error((std::string("batch graph: ") + cudaGetErrorString(e)).c_str());
      return GA_ERR_CUDA;
    }
    g_batches.push_back(nb);
    bg = &g_batches.back();
  }
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < count && e == cudaSuccess; ++i)
    e = cudaStreamWaitEvent(bg->stream, ctxs[i]->ef ? ctxs[i]->ef->ev[0] : ctxs[i]->ed->ev[0], 0);
  if (e == cudaSuccess) e = cudaGraphLaunch(bg->exec, bg->stream);
  if (e == cudaSuccess) e = cudaEventRecord(bg->done, bg->stream);
  if (e != cudaSuccess) {
    ga::set_global_error((std::string("batch launch: ") + cudaGetErrorString(e)).c_str());
    return GA_ERR_CUDA;
  }
  for (int i = 0; i < count; ++i) {
    ga_ctx* c = ctxs[i];
    const auto t0 = std::chrono::steady_clock::now();
    st[i] = dispatch(c, [&](auto& en) {
      en.ck(cudaStreamWaitEvent(en.st, bg->done, 0), "wait");
      en.ck(cudaEventRecord(en.ev[1], en.st), "event");
      en.res_complete();
      stage_out(en, v[i], en.current(), en.vl, mem);
    });
    c->stats.t_total_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (st[i] == GA_OK && !c->stats.converged) st[i] = GA_ERR_NOT_CONVERGED;
    if (stats) stats[i] = c->stats;
  }
  return batch_status(count, ctxs, st);
}

ga_status ga_solve_batch(int count, ga_ctx* const* ctxs, void* const* v, int mem, ga_stats* stats) {
  if (count < 0 || (count > 0 && (!ctxs || !v))) return GA_ERR_ARG;
  for (int i = 0; i < count; ++i)
    if (!ctxs[i] || !v[i]) return GA_ERR_ARG;
  bool all_resident = count > 0;
  for (int i = 0; i < count; ++i) all_resident = all_resident && ctxs[i]->opts.graphs == 2;
  if (all_resident) return solve_batch_resident(count, ctxs, v, mem, stats);
  // Each problem is solved by its own host worker on its own context stream, so the kernels of
  // different problems overlap on the GPU while any one of them waits for a line-search decision.
  int dev = 0;
  cudaGetDevice(&dev);
  std::vector<ga_status> st(count, GA_OK);
  std::atomic<int> next{0};
  const unsigned hw = std::thread::hardware_concurrency();
  const int nworkers = std::max(1, std::min(count, (int)std::min(32u, hw ? hw : 8u)));
  auto worker = [&] {
    cudaSetDevice(dev);
    for (int i = next.fetch_add(1); i < count; i = next.fetch_add(1))
      st[i] = ga_solve(ctxs[i], v[i], mem, stats ? &stats[i] : nullptr);
  };
  std::vector<std::thread> pool;
  for (int t = 1; t < nworkers; ++t) pool.emplace_back(worker);
  worker();
  for (auto& th : pool) th.join();
  return batch_status(count, ctxs, st);
}

// ---- operator-level entry points (ga_ops.h) --------------------------------------------------------

ga_status ga_op_departure(ga_ctx* ctx, const void* v, void* xm, void* xp) {
  if (!ctx || !v || !xm || !xp) return GA_ERR_ARG;
  return dispatch(ctx, [&](auto& e) {
    using T = typename std::remove_reference<decltype(*e.m0)>::type;
    e.ck(launch_departure<T>(e.g, static_cast<const T*>(v), static_cast<T*>(xm), static_cast<T*>(xp), (T)e.ht,
                             e.st), "departure");
    e.ck(cudaStreamSynchronize(e.st), "sync");
  });
}

ga_status ga_op_forward(ga_ctx* ctx, const void* v, void* states) {
  if (!ctx || !v || !states) return GA_ERR_ARG;
  return dispatch(ctx, [&](auto& e) {
    using T = typename std::remove_reference<decltype(*e.m0)>::type;
    const T* vv = static_cast<const T*>(v);
    T* out = static_cast<T*>(states);
    e.compute_mu(vv);
    e.ck(launch_departure<T>(e.g, vv, e.xm, e.xp, (T)e.ht, e.st), "departure");
    e.ck(cudaMemcpyAsync(out, e.m0, sizeof(T) * e.nv, cudaMemcpyDeviceToDevice, e.st), "copy");
    e.chain_reset();
    for (int j = 0; j < e.nt; ++j) e.sl_forward(out + (long long)j * e.nv, out + (long long)(j + 1) * e.nv);
    e.ck(cudaStreamSynchronize(e.st), "sync");
  });
}

ga_status ga_op_adjoint(ga_ctx* ctx, const void* v, const void* lam1, void* lams) {
  if (!ctx || !v || !lam1 || !lams) return GA_ERR_ARG;
  return dispatch(ctx, [&](auto& e) {
    using T = typename std::remove_reference<decltype(*e.m0)>::type;
    const T* vv = static_cast<const T*>(v);
    T* out = static_cast<T*>(lams);
    e.compute_mu(vv);
    e.ck(launch_departure<T>(e.g, vv, e.xm, e.xp, (T)e.ht, e.st), "departure");
    const long long nv = e.nv;
    e.ck(cudaMemcpyAsync(out + (long long)e.nt * nv, lam1, sizeof(T) * nv, cudaMemcpyDeviceToDevice, e.st), "copy");
    e.adjoint_chain_reset();
    for (int j = e.nt - 1; j >= 0; --j) e.sl_adjoint(out + (long long)(j + 1) * nv, out + (long long)j * nv);
    e.ck(cudaStreamSynchronize(e.st), "sync");
  });
}

ga_status ga_op_body_force(ga_ctx* ctx, const void* v, const void* lam1, void* b) {
  if (!ctx || !v || !lam1 || !b) return GA_ERR_ARG;
  return dispatch(ctx, [&](auto& e) {
    using T = typename std::remove_reference<decltype(*e.m0)>::type;
    const T* vv = static_cast<const T*>(v);
    e.compute_mu(vv);
    e.ck(launch_departure<T>(e.g, vv, e.xm, e.xp, (T)e.ht, e.st), "departure");
    e.forward_all();
    e.ck(cudaMemcpyAsync(e.lam[0], lam1, sizeof(T) * e.nv, cudaMemcpyDeviceToDevice, e.st), "copy");
    e.body_force(e.lam[0]);
    e.ck(cudaMemcpyAsync(b, e.body, sizeof(T) * e.vl, cudaMemcpyDeviceToDevice, e.st), "copy");
    e.ck(cudaStreamSynchronize(e.st), "sync");
  });
}

ga_status ga_op_deriv(ga_ctx* ctx, const void* f, int axis, void* df) {
  if (!ctx || !f || !df || f == df) return GA_ERR_ARG;
  if (axis < 0 || axis >= ctx->desc.dim) return GA_ERR_ARG;
  return dispatch(ctx, [&](auto& e) {
    using T = typename std::remove_reference<decltype(*e.m0)>::type;
    e.deriv(e.g.axis_of(axis), static_cast<const T*>(f), nullptr, static_cast<T*>(df), 1.0, false);
    e.ck(cudaStreamSynchronize(e.st), "sync");
  });
}

// pencils[c] (c < dim): one-field passes along axis c; pencils[dim + c]: two-time-step passes.
ga_status ga_op_get_tiles(const ga_ctx* ctx, int* pencils) {
  if (!ctx || !pencils) return GA_ERR_ARG;
  const int dim = ctx->desc.dim;
  for (int pair = 0; pair < 2; ++pair)
    for (int c = 0; c < dim; ++c) {
      const int a = 3 - dim + c;
      const int L = ctx->desc.n[c];
      const int p = ctx->ef ? (pair ? ctx->ef->ft.pair_pencils[a] : ctx->ef->ft.deriv_pencils[a])
                            : (pair ? ctx->ed->ft.pair_pencils[a] : ctx->ed->ft.deriv_pencils[a]);
      pencils[pair * dim + c] =
          L == ga::kRegFftLen
              ? ga::kRegFftPencils
              : (p > 0 ? p : (ctx->ef ? ga::deriv_default_pencils<float>(L) : ga::deriv_default_pencils<double>(L)));
    }
  return GA_OK;
}

ga_status ga_op_get_sl_depth(const ga_ctx* ctx, int* state_depth, int* adjoint_depth) {
  if (!ctx || !state_depth || !adjoint_depth) return GA_ERR_ARG;
  const ga::Grid& g = ctx->ef ? ctx->ef->g : ctx->ed->g;
  *state_depth = g.sl_bz;
  *adjoint_depth = g.sl_bz_adj;
  return GA_OK;
}

ga_status ga_op_set_sl_depth(ga_ctx* ctx, int state_depth, int adjoint_depth) {
  if (!ctx) return GA_ERR_ARG;
  int d[2] = {state_depth == 0 ? 8 : state_depth, adjoint_depth == 0 ? 8 : adjoint_depth};
  for (int i = 0; i < 2; ++i) {
    bool known = false;
    for (int k : ga::kSlDepths) known = known || k == d[i];
    if (!known) {
      set_err(ctx, "ga_op_set_sl_depth: brick depth %d is not one of 4, 8, 12", d[i]);
      return GA_ERR_ARG;
    }
  }
  ga::Grid& g = ctx->ef ? ctx->ef->g : ctx->ed->g;
  g.sl_bz = d[0];
  g.sl_bz_adj = d[1];
  return GA_OK;
}

ga_status ga_op_set_tiles(ga_ctx* ctx, const int* pencils) {
  if (!ctx || !pencils) return GA_ERR_ARG;
  const int dim = ctx->desc.dim;
  for (int i = 0; i < 2 * dim; ++i) {
    const int L = ctx->desc.n[i % dim];
    const bool fits = ctx->ef ? ga::deriv_pencils_fit<float>(L, pencils[i]) : ga::deriv_pencils_fit<double>(L, pencils[i]);
    if (pencils[i] < 0 || (pencils[i] > 0 && !fits)) {
      set_err(ctx, "ga_op_set_tiles: %d pencils per CTA along axis %d do not fit", pencils[i], i % dim);
      return GA_ERR_ARG;
    }
  }
  for (int i = 0; i < 2 * dim; ++i) {
    const int a = 3 - dim + i % dim;
    int* dst = ctx->ef ? (i < dim ? ctx->ef->ft.deriv_pencils : ctx->ef->ft.pair_pencils)
                       : (i < dim ? ctx->ed->ft.deriv_pencils : ctx->ed->ft.pair_pencils);
    dst[a] = pencils[i];
  }
  return GA_OK;
}

ga_status ga_op_div(ga_ctx* ctx, const void* v, void* mu) {
  if (!ctx || !v || !mu) return GA_ERR_ARG;
  return dispatch(ctx, [&](auto& e) {
    using T = typename std::remove_reference<decltype(*e.m0)>::type;
    e.compute_mu(static_cast<const T*>(v));
    e.ck(cudaMemcpyAsync(mu, e.mu, sizeof(T) * e.nv, cudaMemcpyDeviceToDevice, e.st), "copy");
    e.ck(cudaStreamSynchronize(e.st), "sync");
  });
}

ga_status ga_op_fft_r2c(ga_ctx* ctx, const void* f, void* fhat) {
  if (!ctx || !f || !fhat) return GA_ERR_ARG;
  return dispatch(ctx, [&](auto& e) {
    using T = typename std::remove_reference<decltype(*e.m0)>::type;
    e.r2c(static_cast<const T*>(f), static_cast<cx<T>*>(fhat));
    e.ck(cudaStreamSynchronize(e.st), "sync");
  });
}

ga_status ga_op_fft_c2r(ga_ctx* ctx, const void* fhat, void* f) {
  if (!ctx || !fhat || !f) return GA_ERR_ARG;
  return dispatch(ctx, [&](auto& e) {
    using T = typename std::remove_reference<decltype(*e.m0)>::type;
    e.ck(cudaMemcpyAsync(e.bh, fhat, sizeof(cx<T>) * e.g.nhalf, cudaMemcpyDeviceToDevice, e.st), "copy");
    e.c2r(e.bh, static_cast<T*>(f));
    e.ck(cudaStreamSynchronize(e.st), "sync");
  });
}

ga_status ga_op_apply_L(ga_ctx* ctx, const void* v, void* Lv) {
  if (!ctx || !v || !Lv) return GA_ERR_ARG;
  return dispatch(ctx, [&](auto& e) {
    using T = typename std::remove_reference<decltype(*e.m0)>::type;
    const T* vv = static_cast<const T*>(v);
    for (int c = 0; c < e.dim; ++c) e.r2c(vv + c * e.nv, e.bh + c * e.g.nhalf);
    SpecArgs sa{SPEC_APPLY_L, e.s, e.alpha, 0};
    e.ck(launch_spectral<T>(e.g, sa, e.bh, e.st), "spectral");
    for (int c = 0; c < e.dim; ++c) e.c2r(e.bh + c * e.g.nhalf, static_cast<T*>(Lv) + c * e.nv);
    e.ck(cudaStreamSynchronize(e.st), "sync");
  });
}

ga_status ga_op_leray(ga_ctx* ctx, const void* v, void* pv) {
  if (!ctx || !v || !pv) return GA_ERR_ARG;
  return dispatch(ctx, [&](auto& e) {
    using T = typename std::remove_reference<decltype(*e.m0)>::type;
    const T* vv = static_cast<const T*>(v);
    for (int c = 0; c < e.dim; ++c) e.r2c(vv + c * e.nv, e.bh + c * e.g.nhalf);
    SpecArgs sa{SPEC_LERAY, e.s, e.alpha, 1};
    e.ck(launch_spectral<T>(e.g, sa, e.bh, e.st), "spectral");
    for (int c = 0; c < e.dim; ++c) e.c2r(e.bh + c * e.g.nhalf, static_cast<T*>(pv) + c * e.nv);
    e.ck(cudaStreamSynchronize(e.st), "sync");
  });
}

ga_status ga_op_dots(ga_ctx* ctx, const void* a, const void* const* b, int count, size_t len, double* out) {
  if (!ctx || !a || !b || !out || count < 1 || count > kMaxDots || len < 1) return GA_ERR_ARG;
  return dispatch(ctx, [&](auto& e) {
    using T = typename std::remove_reference<decltype(*e.m0)>::type;
    std::vector<const T*> bl(count);
    for (int i = 0; i < count; ++i) bl[i] = static_cast<const T*>(b[i]);
    e.ck(launch_dots<T>(static_cast<const T*>(a), bl.data(), count, (long long)len, e.dpart, e.dres + kResDots, e.st),
         "dots");
    e.read_results(kResDots + count);
    for (int i = 0; i < count; ++i) out[i] = e.hres[kResDots + i];
  });
}

ga_status ga_op_lsq(ga_ctx* ctx, int m, double c, const double* a, const double* M, double* beta) {
  if (!ctx || !a || !M || !beta || m < 1 || m > kMaxWin) return GA_ERR_ARG;
  return dispatch(ctx, [&](auto& e) {
    std::vector<double> h(1 + m + m * m + m);
    h[0] = c;
    for (int i = 0; i < m; ++i) h[1 + i] = a[i];
    double* dd = e.dpart;  // scratch: dots at 0, M at 1 + m, beta after
    e.ck(cudaMemcpyAsync(dd, h.data(), sizeof(double) * (1 + m), cudaMemcpyHostToDevice, e.st), "copy");
    e.ck(cudaMemcpyAsync(dd + 1 + m, M, sizeof(double) * m * m, cudaMemcpyHostToDevice, e.st), "copy");
    e.ck(launch_lsq(m, dd, dd + 1 + m, m, dd + 1 + m + m * m, nullptr, e.st), "lsq");
    e.ck(cudaMemcpyAsync(beta, dd + 1 + m + m * m, sizeof(double) * m, cudaMemcpyDeviceToHost, e.st), "copy");
    e.ck(cudaStreamSynchronize(e.st), "sync");
  });
}

ga_status ga_transport(ga_ctx* ctx, const void* v, void* m1_out, int mem) {
  if (!ctx || !v || !m1_out || (mem != GA_MEM_HOST && mem != GA_MEM_DEVICE)) return GA_ERR_ARG;
  return dispatch(ctx, [&](auto& e) {
    auto* vin = stage_in(e, v, e.vl, mem, e.io_a);
    if (e.needs_mu_forward()) e.compute_mu(vin);
    const auto* mT = e.forward_final(vin);
    stage_out(e, m1_out, mT, e.nv, mem);
  });
}

ga_status ga_transport_vjp(ga_ctx* ctx, const void* v, const void* gamma, void* grad_v, int mem) {
  if (!ctx || !v || !gamma || !grad_v || (mem != GA_MEM_HOST && mem != GA_MEM_DEVICE)) return GA_ERR_ARG;
  return dispatch(ctx, [&](auto& e) {
    using T = typename std::remove_reference<decltype(*e.m0)>::type;
    auto* vin = stage_in(e, v, e.vl, mem, e.io_a);
    const T* gam = stage_in(e, gamma, e.nv, mem, e.lam[0]);
    if (gam != e.lam[0])
      e.ck(cudaMemcpyAsync(e.lam[0], gam, sizeof(T) * e.nv, cudaMemcpyDeviceToDevice, e.st), "copy");
    e.compute_mu(vin);
    e.ck(launch_departure<T>(e.g, vin, e.xm, e.xp, (T)e.ht, e.st), "departure");
    e.forward_all();
    e.body_force(e.lam[0]);
    // grad_v = -b
    e.ck(launch_axpy<T>(e.io_b, e.body, e.body, -2.0, e.vl, e.st), "negate");
    stage_out(e, grad_v, e.io_b, e.vl, mem);
  });
}

ga_status ga_transport_vjp_exact(ga_ctx* ctx, const void* v, const void* gamma, void* grad_v, int mem) {
  if (!ctx || !v || !gamma || !grad_v || (mem != GA_MEM_HOST && mem != GA_MEM_DEVICE)) return GA_ERR_ARG;
  return dispatch(ctx, [&](auto& e) {
    using T = typename std::remove_reference<decltype(*e.m0)>::type;
    e.dto_require_advection("ga_transport_vjp_exact");
    auto* vin = stage_in(e, v, e.vl, mem, e.io_a);
    const T* gam = stage_in(e, gamma, e.nv, mem, e.lam[0]);
    e.dto_forward(vin);
    e.dto_backward(vin, gam, 1.0, e.io_b);
    stage_out(e, grad_v, e.io_b, e.vl, mem);
  });
}

// ---- event timing of one kernel class over a region (used by the benchmark) --------------------------
long long ga_kernel_launches(void) { return ga::g_launches.load(std::memory_order_relaxed); }

ga_status ga_prof_start(ga_ctx* ctx, int kernel_class) {
  if (!ctx || kernel_class < 0 || kernel_class > 4) return GA_ERR_ARG;
  return dispatch(ctx, [&](auto& e) {
    if (e.prof_ev.empty()) {
      e.prof_ev.resize(4096);
      for (auto& ev : e.prof_ev) e.ck(cudaEventCreate(&ev), "cudaEventCreate");
    }
    e.prof_class = kernel_class;
    e.prof_used = 0;
    e.prof_ms = 0.0;
    e.prof_launches = 0;
  });
}

ga_status ga_prof_stop(ga_ctx* ctx, double* total_ms, long long* launches) {
  if (!ctx || !total_ms || !launches) return GA_ERR_ARG;
  return dispatch(ctx, [&](auto& e) {
    e.prof_flush();
    *total_ms = e.prof_ms;
    *launches = e.prof_launches;
    e.prof_class = -1;
  });
}

}  // extern "C"
