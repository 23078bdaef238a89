// reg.cu -- context, transport sweeps, reduced-space operators and the
// inexact Gauss-Newton-Krylov solve behind the C ABI of include/reg.h
// (Mang & Biros, arXiv:1408.6299: Alg. 1 outer iteration, Alg. 2 Hessian
// matvec, Sec. 3.2-3.3 discretisation and preconditioning).
//
// Time stepping is Heun's RK2 on the nodes t_j = j/n_t. A sweep reads the
// velocity v(t_j) = sum_l T_l(2 t_j - 1) v_l (Sec. 3.3.2) at the two nodes of a
// step. The state gradients grad m_j are either stored for every node
// (ckpt_every = 0) or recomputed segment by segment from every K-th state
// (ckpt_every = K). The body-force time integral uses the trapezoid rule on
// the nodes (default) or the stage values of the discrete adjoint.
#include <chrono>
#include <functional>
#include <cfloat>
#include <cmath>
#include <cstring>
#include <map>
#include <thread>
#include <tuple>
#include <memory>
#include <numeric>
#include <new>
#include <string>
#include <vector>

#include "../../include/reg.h"
#include "internal.h"
#include "fused.cuh"
#include "pointwise.h"

using namespace reg;

namespace {

thread_local std::string g_create_error;

// device buffer owned by the context
template <typename T>
struct DBuf {
  T* p = nullptr;
  size_t n = 0;
  DBuf() = default;
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  ~DBuf() { release(); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
  T* get(size_t count) {
    if (count <= n && p) return p;
    release();
    cudaError_t e = cudaMalloc(&p, count * sizeof(T));
    if (e != cudaSuccess) {
      p = nullptr;
      (void)cudaGetLastError();
      throw StatusError{REG_ENOMEM, "device allocation of " + std::to_string(count * sizeof(T)) + " bytes failed"};
    }
    n = count;
    return p;
  }
};

// Chebyshev polynomials T_l(x) by the three-term recurrence
void cheb_values(int nc, double t, double* b) {
  double x = 2.0 * t - 1.0;
  for (int l = 0; l < nc; ++l) b[l] = l == 0 ? 1.0 : (l == 1 ? x : 2.0 * x * b[l - 1] - b[l - 2]);
}

// exact int_0^1 T_a(2t-1) T_b(2t-1) dt via T_a T_b = (T_{a+b} + T_{|a-b|})/2
double cheb_gram_entry(int a, int b) {
  auto I = [](int m) { return (m % 2) ? 0.0 : 2.0 / (1.0 - (double)m * (double)m); };
  return 0.25 * (I(a + b) + I(a > b ? a - b : b - a));
}

bool invert_small(int n, const std::vector<double>& A, std::vector<double>& Ai) {
  std::vector<double> M(n * 2 * n);
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < 2 * n; ++c) M[r * 2 * n + c] = c < n ? A[r * n + c] : (c - n == r ? 1.0 : 0.0);
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(M[r * 2 * n + c]) > std::fabs(M[piv * 2 * n + c])) piv = r;
    if (M[piv * 2 * n + c] == 0.0) return false;
    for (int k = 0; k < 2 * n; ++k) std::swap(M[c * 2 * n + k], M[piv * 2 * n + k]);
    double p = M[c * 2 * n + c];
    for (int k = 0; k < 2 * n; ++k) M[c * 2 * n + k] /= p;
    for (int r = 0; r < n; ++r)
      if (r != c) {
        double f = M[r * 2 * n + c];
        for (int k = 0; k < 2 * n; ++k) M[r * 2 * n + k] -= f * M[c * 2 * n + k];
      }
  }
  Ai.assign(n * n, 0.0);
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < n; ++c) Ai[r * n + c] = M[r * 2 * n + n + c];
  return true;
}

// per-precision scratch of the sweeps
template <typename T>
struct Work {
  using C = cx<T>;
  DBuf<C> U, W, X;         // spectra
  DBuf<C> U2, W2, X2;      // spectra of the second field of a two-field stage
  DBuf<T> yhS, accS, srcS; // state stage values and one source of the fused forward sweep
  DBuf<T> G, q, va, vb, wa, wb;  // d fields
  DBuf<T> m, yh, acc, k, lam;    // fields
  DBuf<T> vcoef, wcoef;          // coefficient vectors in precision T
  DBuf<T> gm, gmh, ck;           // state gradients (all nodes or one segment), stage gradients, checkpoints
  DBuf<T> fhi, flo;              // single precision body force as a compensated pair
  DBuf<T> src;                   // source grad m_j . v~(t_j) per node (all nodes or one segment)
  DBuf<T> mtil, lamN, yh2, acc2, st0, st1, Gt, mR, m1;  // full Newton matvec
};

}  // namespace

struct reg_ctx {
  int d = 0, n_t = 0, n_c = 0, rtype = 1, stokes = 0, prec = 0, ckpt = 0, quad = 0;
  int hess = 0;  // REG_HESS_GN or REG_HESS_NEWTON
  // stacked problems (g.B > 1): one beta per problem, per-problem reductions
  std::vector<double> betas;
  DBuf<double> betas_dev, seg_scr, coefA, coefC, sv_v;
  double beta = 0;
  cudaStream_t s = nullptr;
  Grid g;
  double hd = 1.0;  // cell volume
  std::string err;

  std::vector<double> bnode;  // (n_t+1) x n_c basis values at the nodes
  std::vector<double> Cg, Ci;
  DBuf<double> Cg_dev, Ci_dev;

  std::unique_ptr<Spectral<double>> sp64;
  std::unique_ptr<Spectral<float>> sp32;
  Work<double> w64;
  Work<float> w32;

  DBuf<double> mT, mR;
  bool have_images = false;
  bool ready = false;  // linearisation point set (stored state valid)
  DBuf<double> vlin;   // linearisation point

  DBuf<double> f;      // body force (n_c d N)
  DBuf<double2> SV, SF;  // spectra of coefficient vectors for the tail
  DBuf<double> red;    // reduction scratch
  DBuf<double> tmpA, tmpB;  // coefficient-vector temporaries
  DBuf<double> stage_in[3], stage_out;  // staging of host arrays
  // det F scratch
  DBuf<double> F, Fh, K1, K2, gvl, gvt, det, ang;
  DBuf<double> disp_src;                          // sources -v_i(t) of the deformation map
  DBuf<double> lz_q, lz_u, lz_up, lz_w, lz_z;     // Lanczos vectors
  DBuf<double> ct_start, ct_good;                 // continuation iterates
  // solve vectors
  DBuf<double> sv_g, sv_s, sv_r, sv_z, sv_p, sv_Hp, sv_vt;
  KernelProfiler prof;  // CUDA-event bracketing of launches by kind (off unless enabled)
  // CUDA graph of the Hessian matvec (contexts with their own stream): the
  // sweeps and the tail read the direction from gdir and write gout
  bool graphs = false;
  cudaGraphExec_t gexec = nullptr;
  size_t gsig = 0;
  long gkernels = 0;
  DBuf<double> gdir, gout;
  // device-driven lockstep loops (stacked problems): per-problem scalars, the
  // control block, and the graphs of the PCG and line-search loops
  DBuf<double> lk;
  DBuf<int> lkc;
  std::vector<double> lkh;
  cudaGraphExec_t lk_pcg = nullptr, lk_ls = nullptr;
  size_t lk_sig = 0;
  int lk_state = 0;  // 0 not built yet, 1 built, -1 refused (host-driven loops)
  ~reg_ctx() {
    if (gexec) cudaGraphExecDestroy(gexec);
    if (lk_pcg) cudaGraphExecDestroy(lk_pcg);
    if (lk_ls) cudaGraphExecDestroy(lk_ls);
  }

  long N() const { return g.N; }
  long ncdN() const { return (long)n_c * d * g.N; }
  long dN() const { return (long)d * g.N; }
  double h() const { return 1.0 / n_t; }
  Coefs basis_at_node(int j, double scale = 1.0) const {
    Coefs c{};
    for (int l = 0; l < n_c; ++l) c.c[l] = scale * bnode[(size_t)j * n_c + l];
    return c;
  }
  double trap_w(int j) const { return (j == 0 || j == n_t) ? 0.5 * h() : h(); }
};

namespace {

// ---------------------------------------------------------------------------
// host/device pointer handling
// ---------------------------------------------------------------------------
// true for memory the kernels can address directly (device memory of the
// current device, or managed memory), false for host memory (staged through
// the context's buffers); device memory of another device is refused, since
// kernels launched on the current device would fault on it
bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  if (a.type != cudaMemoryTypeDevice) return false;
  int dev = 0;
  REG_CUDA(cudaGetDevice(&dev));
  if (a.device != dev)
    throw StatusError{REG_EINVAL, "array argument lives on device " + std::to_string(a.device) + " but device " +
                                      std::to_string(dev) + " is current"};
  return true;
}

const double* input_ptr(reg_ctx* c, const double* p, long n, int slot) {
  if (!p) throw StatusError{REG_EINVAL, "null array argument"};
  if (is_device_ptr(p)) return p;
  double* d = c->stage_in[slot].get(n);
  REG_CUDA(cudaMemcpyAsync(d, p, n * sizeof(double), cudaMemcpyHostToDevice, c->s));
  return d;
}

struct Output {
  reg_ctx* c;
  double* user;
  double* dev;
  long n;
  bool host;
  Output(reg_ctx* c_, double* p, long n_, DBuf<double>& stage) : c(c_), user(p), n(n_) {
    if (!p) throw StatusError{REG_EINVAL, "null output argument"};
    host = !is_device_ptr(p);
    dev = host ? stage.get(n) : p;
  }
  void finish() {
    if (host) REG_CUDA(cudaMemcpyAsync(user, dev, n * sizeof(double), cudaMemcpyDeviceToHost, c->s));
    REG_CUDA(cudaStreamSynchronize(c->s));
  }
};

template <typename T>
Work<T>& work(reg_ctx* c);
template <>
Work<double>& work<double>(reg_ctx* c) { return c->w64; }
template <>
Work<float>& work<float>(reg_ctx* c) { return c->w32; }
template <typename T>
Spectral<T>& spectral(reg_ctx* c);
template <>
Spectral<double>& spectral<double>(reg_ctx* c) { return *c->sp64; }
template <>
Spectral<float>& spectral<float>(reg_ctx* c) {
  if (!c->sp32) c->sp32.reset(new Spectral<float>(c->g, c->s));
  return *c->sp32;
}

template <typename T>
void grad_into(reg_ctx* c, const T* u, T* G) {
  Work<T>& w = work<T>(c);
  spectral<T>(c).grad(u, G, w.U.get(c->g.Nc), w.W.get(c->g.Nc));
}

// velocity (coefficients in precision T) at node j: a pointer to d fields
template <typename T>
const T* vel_node(reg_ctx* c, const T* coef, int j, T* buf) {
  if (c->n_c == 1) return coef;
  vel_at<T, T>(coef, c->n_c, c->basis_at_node(j), buf, c->dN(), c->s);
  return buf;
}

// fused advection stage on u: k = -a.grad u [- gm.w], Heun stage update.
// u_ready: w.U already holds the spectrum of u (left there by the previous
// stage); emit: leave the spectrum of out1 in w.U for the next stage;
// spec_only: out1 is needed only as that spectrum (no real store).
template <typename T>
void adv(reg_ctx* c, const T* u, const T* a, const T* gm, const T* wv, const T* y, T* out1, T* out2, T* Gkeep,
         int stage, const T* src = nullptr, const T* sw = nullptr, T* Sout = nullptr, bool u_ready = false,
         bool emit = false, bool spec_only = false) {
  Work<T>& w = work<T>(c);
  const long N = c->N(), Nc = c->g.Nc;
  fused::AdvEpi<T> e{};
  for (int i = 0; i < c->d; ++i) {
    e.a[i] = a ? a + i * N : nullptr;
    e.gm[i] = gm ? gm + i * N : nullptr;
    e.w[i] = gm ? wv + i * N : nullptr;
    e.G[i] = Gkeep ? Gkeep + i * N : nullptr;
    e.sw[i] = sw ? sw + i * N : nullptr;
  }
  e.src = src;
  e.Sout = Sout;
  e.y = y;
  e.out1 = out1;
  e.out2 = out2;
  e.h = (T)c->h();
  e.stage = stage;
  e.out1_spectral_only = spec_only ? 1 : 0;
  adv_stage<T>(spectral<T>(c), u, e, w.U.get(Nc), w.W.get(Nc), w.X.get(Nc), u_ready, emit);
}

// epilogue of an advection stage without stored-gradient source terms
template <typename T>
fused::AdvEpi<T> adv_epi(reg_ctx* c, const T* a, const T* y, T* out1, T* out2, int stage, const T* src = nullptr,
                         const T* sw = nullptr, T* Sout = nullptr) {
  const long N = c->N();
  fused::AdvEpi<T> e{};
  for (int i = 0; i < c->d; ++i) {
    e.a[i] = a ? a + i * N : nullptr;
    e.sw[i] = sw ? sw + i * N : nullptr;
  }
  e.src = src;
  e.Sout = Sout;
  e.y = y;
  e.out1 = out1;
  e.out2 = out2;
  e.h = (T)c->h();
  e.stage = stage;
  return e;
}

// two 3D advection stages sharing their passes
template <typename T>
void adv2(reg_ctx* c, const T* uA, const fused::AdvEpi<T>& eA, const T* uB, const fused::AdvEpi<T>& eB) {
  Work<T>& w = work<T>(c);
  const long Nc = c->g.Nc;
  cx<T>* Z[6] = {w.U.get(Nc), w.W.get(Nc), w.X.get(Nc), w.U2.get(Nc), w.W2.get(Nc), w.X2.get(Nc)};
  adv2_stage<T>(spectral<T>(c), uA, eA, uB, eB, Z);
}

// grad u into G (d fields) through the fused stage passes
template <typename T>
void grad_fused(reg_ctx* c, const T* u, T* G, bool u_ready = false) {
  adv<T>(c, u, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, G, 1, nullptr, nullptr, nullptr, u_ready);
}

// fused divergence stage on lam: k = div(a lam), Heun stage update; e carries
// the optional body-force accumulation of stage 1
template <typename T>
void divh(reg_ctx* c, const T* lam, const T* a, const T* y, T* out1, T* out2, int stage,
          fused::DivEpi<T> e = fused::DivEpi<T>{}) {
  Work<T>& w = work<T>(c);
  const long Nc = c->g.Nc;
  e.y = y;
  e.out1 = out1;
  e.out2 = out2;
  e.h = (T)c->h();
  e.stage = stage;
  div_stage<T>(spectral<T>(c), lam, a, e, w.U.get(Nc), w.W.get(Nc), w.X.get(Nc));
}

// ---------------------------------------------------------------------------
// State solve (Eq. first-order-forward), steps j0..j1-1 from the state in w.m.
//   gm  (optional): grad m_j into slot (j - base) for j = j0..j1 (the last slot
//                   is the extra gradient of the final state)
//   gmh (optional): grad of the stage-2 input of step j into slot (j+1 - base)
//   ck  (optional): m_j into slot j/K for j % K == 0 (and the final state)
// ---------------------------------------------------------------------------
template <typename T>
void state_steps(reg_ctx* c, const T* vcoef, int j0, int j1, T* gm, T* gmh, int base, T* ck) {
  Work<T>& w = work<T>(c);
  const long N = c->N(), dN = c->dN();
  const T h = (T)c->h();
  T* m = w.m.get(N);
  T* yh = w.yh.get(N);
  T* acc = w.acc.get(N);
  T* G = w.G.get(dN);
  T* va = w.va.get(dN);
  T* vb = w.vb.get(dN);
  // each stage leaves the spectrum of its out1 in w.U for the next one; the
  // predictor yh is needed only as that spectrum
  bool ready = false;
  for (int j = j0; j < j1; ++j) {
    if (ck && c->ckpt > 0 && j % c->ckpt == 0)
      REG_CUDA(cudaMemcpyAsync(ck + (long)(j / c->ckpt) * N, m, N * sizeof(T), cudaMemcpyDeviceToDevice, c->s));
    adv<T>(c, m, vel_node<T>(c, vcoef, j, va), nullptr, nullptr, m, yh, acc, gm ? gm + (long)(j - base) * dN : nullptr,
           1, nullptr, nullptr, nullptr, ready, true, true);
    const bool more = j + 1 < j1 || gm;  // the spectrum of m is read next
    adv<T>(c, yh, vel_node<T>(c, vcoef, j + 1, vb), nullptr, nullptr, acc, m, nullptr,
           gmh ? gmh + (long)(j + 1 - base) * dN : nullptr, 2, nullptr, nullptr, nullptr, true, more);
    ready = more;
  }
  if (ck && c->ckpt > 0 && j1 % c->ckpt == 0)
    REG_CUDA(cudaMemcpyAsync(ck + (long)(j1 / c->ckpt) * N, m, N * sizeof(T), cudaMemcpyDeviceToDevice, c->s));
  if (gm) grad_fused<T>(c, m, gm + (long)(j1 - base) * dN, ready);
}

// Recompute state gradients of segment [j0, j1] from the checkpoint at j0.
template <typename T>
void recompute_segment(reg_ctx* c, const T* vcoef, int j0, int j1) {
  Work<T>& w = work<T>(c);
  const long N = c->N(), dN = c->dN();
  T* m = w.m.get(N);
  REG_CUDA(cudaMemcpyAsync(m, w.ck.p + (long)(j0 / c->ckpt) * N, N * sizeof(T), cudaMemcpyDeviceToDevice, c->s));
  state_steps<T>(c, vcoef, j0, j1, w.gm.get((size_t)(c->ckpt + 1) * dN),
                 c->quad ? w.gmh.get((size_t)(c->ckpt + 1) * dN) : nullptr, j0, nullptr);
}

// State re-advance over [j0, j1] from the checkpoint at j0 that keeps, instead
// of the state gradients, the source s_j = grad m_j . w(t_j) of the
// incremental state equation (slot j - j0); w: incremental velocity coefficients.
template <typename T>
void recompute_segment_src(reg_ctx* c, const T* vcoef, const T* wcoef, int j0, int j1) {
  Work<T>& w = work<T>(c);
  const long N = c->N(), dN = c->dN();
  T* m = w.m.get(N);
  T* yh = w.yh.get(N);
  T* acc = w.acc.get(N);
  T* va = w.va.get(dN);
  T* vb = w.vb.get(dN);
  T* wa = w.wa.get(dN);
  T* src = w.src.get((size_t)(c->ckpt + 1) * N);
  REG_CUDA(cudaMemcpyAsync(m, w.ck.p + (long)(j0 / c->ckpt) * N, N * sizeof(T), cudaMemcpyDeviceToDevice, c->s));
  bool ready = false;  // w.U holds the spectrum of m
  for (int j = j0; j < j1; ++j) {
    adv<T>(c, m, vel_node<T>(c, vcoef, j, va), nullptr, nullptr, m, yh, acc, nullptr, 1, nullptr,
           vel_node<T>(c, wcoef, j, wa), src + (long)(j - j0) * N, ready, true, true);
    adv<T>(c, yh, vel_node<T>(c, vcoef, j + 1, vb), nullptr, nullptr, acc, m, nullptr, nullptr, 2, nullptr, nullptr,
           nullptr, true, true);
    ready = true;
  }
  adv<T>(c, m, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, 1, nullptr,
         vel_node<T>(c, wcoef, j1, wa), src + (long)(j1 - j0) * N, ready);
}

// Gradient slots available for node j (after ensure_segment)
template <typename T>
const T* gm_slot(reg_ctx* c, int j, int base) {
  return work<T>(c).gm.p + (long)(j - base) * c->dN();
}
template <typename T>
const T* gmh_slot(reg_ctx* c, int j, int base) {
  return work<T>(c).gmh.p + (long)(j - base) * c->dN();
}

// Full state solve from m0 with storage for later sweeps (store-all or checkpoints).
template <typename T>
void state_solve_store(reg_ctx* c, const T* vcoef, const T* m0) {
  Work<T>& w = work<T>(c);
  const long N = c->N(), dN = c->dN();
  REG_CUDA(cudaMemcpyAsync(w.m.get(N), m0, N * sizeof(T), cudaMemcpyDeviceToDevice, c->s));
  if (c->ckpt == 0) {
    state_steps<T>(c, vcoef, 0, c->n_t, w.gm.get((size_t)(c->n_t + 1) * dN),
                   c->quad ? w.gmh.get((size_t)(c->n_t + 1) * dN) : nullptr, 0, nullptr);
  } else {
    state_steps<T>(c, vcoef, 0, c->n_t, nullptr, nullptr, 0, w.ck.get((size_t)(c->n_t / c->ckpt + 1) * N));
  }
}

// Adjoint solve (Eq. first-order-adjoint) backward from lam (in w.lam at n_t),
// accumulating the body force f_l = int b_l lam grad m dt into f (double).
// The force terms of each step are added in the first stage of the step: the
// trapezoid term of node j+1, or the two stage terms of the discrete adjoint.
// Single precision sweeps accumulate into a compensated pair of floats that is
// converted to double at the end. Leaves lam_0 in w.lam.
template <typename T>
void adjoint_solve(reg_ctx* c, const T* vcoef, double* f) {
  Work<T>& w = work<T>(c);
  const long N = c->N(), dN = c->dN();
  const double hd = c->h();
  T* lam = w.lam.p;
  T* yh = w.yh.get(N);
  T* acc = w.acc.get(N);
  T* va = w.va.get(dN);
  T* vb = w.vb.get(dN);
  T* fhi;
  T* flo = nullptr;
  if (sizeof(T) == sizeof(double)) {
    fhi = reinterpret_cast<T*>(f);
  } else {
    fhi = w.fhi.get(c->ncdN());
    flo = w.flo.get(c->ncdN());
    REG_CUDA(cudaMemsetAsync(flo, 0, c->ncdN() * sizeof(T), c->s));
  }
  REG_CUDA(cudaMemsetAsync(fhi, 0, c->ncdN() * sizeof(T), c->s));
  const int K = c->ckpt > 0 ? c->ckpt : c->n_t;
  for (int seg = (c->n_t - 1) / K; seg >= 0; --seg) {
    int j0 = seg * K, j1 = j0 + K;
    int base = 0;
    if (c->ckpt > 0) {
      recompute_segment<T>(c, vcoef, j0, j1);
      base = j0;
    }
    for (int j = j1 - 1; j >= j0; --j) {
      fused::DivEpi<T> e{};
      e.f_hi = fhi;
      e.f_lo = flo;
      e.nc = c->n_c;
      e.d = c->d;
      e.N = N;
      if (!c->quad) {
        e.gmA = gm_slot<T>(c, j + 1, base);
        Coefs a = c->basis_at_node(j + 1, c->trap_w(j + 1));
        for (int l = 0; l < c->n_c; ++l) e.cA[l] = (T)a.c[l];
      } else {
        e.gmA = gmh_slot<T>(c, j + 1, base);
        e.gmB = gm_slot<T>(c, j, base);
        Coefs a = c->basis_at_node(j + 1, 0.5 * hd), b = c->basis_at_node(j, 0.5 * hd);
        for (int l = 0; l < c->n_c; ++l) {
          e.cA[l] = (T)a.c[l];
          e.cB[l] = (T)b.c[l];
        }
      }
      divh<T>(c, lam, vel_node<T>(c, vcoef, j + 1, vb), lam, yh, acc, 1, e);
      divh<T>(c, yh, vel_node<T>(c, vcoef, j, va), acc, lam, nullptr, 2);
    }
    if (j0 == 0 && !c->quad)
      force_acc<T>(fhi, flo, lam, gm_slot<T>(c, 0, base), c->basis_at_node(0, c->trap_w(0)), c->n_c, c->d, N, c->s);
  }
  if (flo) pair_to_double(reinterpret_cast<const float*>(fhi), reinterpret_cast<const float*>(flo), f, c->ncdN(), c->s);
}

// Full Newton incremental adjoint (Eq. sec-order-iadj / sec-order-icontrol,
// trapezoid quadrature): backward from lam~_1 (in w.lam) with the source
// div(v~ lam); the adjoint lam itself is re-advanced alongside from
// lam_1 = m_R - m_1, so no adjoint trajectory is stored. The body force gains
// lam_j grad m~_j, with m~_j kept by the forward sweep. Per step: the
// incremental stage 1 (force of node j+1, source at t_{j+1}), the two adjoint
// stages, the source at t_j, the incremental stage 2.
template <typename T>
void newton_adjoint(reg_ctx* c, const T* vcoef, const T* wcoef, double* f) {
  Work<T>& w = work<T>(c);
  const long N = c->N(), dN = c->dN();
  T* lt = w.lam.p;  // lam~
  T* yh = w.yh.get(N);
  T* acc = w.acc.get(N);
  T* lam = w.lamN.get(N);
  T* yh2 = w.yh2.get(N);
  T* acc2 = w.acc2.get(N);
  T* sA = w.st0.get(N);
  T* sB = w.st1.get(N);
  T* Gt = w.Gt.get(dN);
  T* va = w.va.get(dN);
  T* vb = w.vb.get(dN);
  T* wa = w.wa.get(dN);
  const T* mtil = w.mtil.p;
  T* fhi;
  T* flo = nullptr;
  if (sizeof(T) == sizeof(double)) {
    fhi = reinterpret_cast<T*>(f);
  } else {
    fhi = w.fhi.get(c->ncdN());
    flo = w.flo.get(c->ncdN());
    REG_CUDA(cudaMemsetAsync(flo, 0, c->ncdN() * sizeof(T), c->s));
  }
  REG_CUDA(cudaMemsetAsync(fhi, 0, c->ncdN() * sizeof(T), c->s));
  // lam_1 = m_R - m_1 and the source at t_1
  lincomb_t<T>((T)1, w.mR.p, (T)-1, w.m1.p, lam, N, c->s);
  divh<T>(c, lam, vel_node<T>(c, wcoef, c->n_t, wa), nullptr, sB, nullptr, 0);
  const int K = c->ckpt > 0 ? c->ckpt : c->n_t;
  for (int seg = (c->n_t - 1) / K; seg >= 0; --seg) {
    int j0 = seg * K, j1 = j0 + K;
    int base = 0;
    if (c->ckpt > 0) {
      recompute_segment<T>(c, vcoef, j0, j1);
      base = j0;
    }
    for (int j = j1 - 1; j >= j0; --j) {
      // incremental stage 1 at t_{j+1}, with the force of node j+1
      grad_fused<T>(c, mtil + (long)(j + 1) * N, Gt);
      fused::DivEpi<T> e{};
      e.f_hi = fhi;
      e.f_lo = flo;
      e.nc = c->n_c;
      e.d = c->d;
      e.N = N;
      e.gmA = gm_slot<T>(c, j + 1, base);
      e.gmC = Gt;
      e.yC = lam;
      Coefs a = c->basis_at_node(j + 1, c->trap_w(j + 1));
      for (int l = 0; l < c->n_c; ++l) e.cA[l] = (T)a.c[l];
      e.src = sB;
      const T* vB = vel_node<T>(c, vcoef, j + 1, vb);
      const T* vA = vel_node<T>(c, vcoef, j, va);
      divh<T>(c, lt, vB, lt, yh, acc, 1, e);
      // adjoint step lam_{j+1} -> lam_j
      divh<T>(c, lam, vB, lam, yh2, acc2, 1);
      divh<T>(c, yh2, vA, acc2, lam, nullptr, 2);
      // source at t_j, then incremental stage 2
      divh<T>(c, lam, vel_node<T>(c, wcoef, j, wa), nullptr, sA, nullptr, 0);
      fused::DivEpi<T> e2{};
      e2.src = sA;
      divh<T>(c, yh, vA, acc, lt, nullptr, 2, e2);
      std::swap(sA, sB);  // the source at t_j is the next step's source at t_{j+1}
    }
    if (j0 == 0)  // node 0: m~_0 = 0, so only the Gauss-Newton term
      force_acc<T>(fhi, flo, lt, gm_slot<T>(c, 0, base), c->basis_at_node(0, c->trap_w(0)), c->n_c, c->d, N, c->s);
  }
  if (flo) pair_to_double(reinterpret_cast<const float*>(fhi), reinterpret_cast<const float*>(flo), f, c->ncdN(), c->s);
}

// Incremental state solve forward from 0 (Eq. gauss-newton, first line), then
// the incremental adjoint backward from -m~_1 with the incremental body force.
// With the trapezoid quadrature the source grad m_j . v~(t_j) of every node is
// formed once (during the state re-advance, or from the stored gradients) and
// read as one field by both Heun stages.
template <typename T>
void gn_sweeps(reg_ctx* c, const T* vcoef, const T* wcoef, double* f) {
  Work<T>& w = work<T>(c);
  const long N = c->N(), dN = c->dN();
  const T h = (T)c->h();
  T* y = w.lam.get(N);  // the incremental state ends up as -lam~_1 in place
  T* yh = w.yh.get(N);
  T* acc = w.acc.get(N);
  T* va = w.va.get(dN);
  T* vb = w.vb.get(dN);
  T* wa = w.wa.get(dN);
  T* wb = w.wb.get(dN);
  const bool use_src = !c->quad;
  const int K = c->ckpt > 0 ? c->ckpt : c->n_t;
  T* mtil = nullptr;
  if (c->hess == REG_HESS_NEWTON) {  // keep every node of the incremental state
    mtil = w.mtil.get((size_t)(c->n_t + 1) * N);
    REG_CUDA(cudaMemsetAsync(mtil, 0, N * sizeof(T), c->s));
  }
  if (use_src && c->ckpt == 0) {
    T* src = w.src.get((size_t)(c->n_t + 1) * N);
    for (int j = 0; j <= c->n_t; ++j)
      dot_fields<T>(gm_slot<T>(c, j, 0), vel_node<T>(c, wcoef, j, wa), src + (long)j * N, c->d, N, c->s);
  }
  if (use_src && c->ckpt > 0 && c->d == 3) {
    // Checkpointed 3D sweep: the state re-advance and the incremental sweep
    // share their passes. At each t_j one two-field stage runs the state's
    // stage 1 (with the source s_j = grad m_j . v~(t_j) of its epilogue) and
    // the incremental stage 2 of step j-1 (which takes s_j from the same
    // epilogue); a second one runs the state's stage 2 and the incremental
    // stage 1 of step j (source s_j, kept in one field).
    T* m = w.m.get(N);
    T* yhS = w.yhS.get(N);
    T* accS = w.accS.get(N);
    T* sj = w.srcS.get(N);
    for (int seg = 0; seg * K < c->n_t; ++seg) {
      const int j0 = seg * K, j1 = j0 + K;
      REG_CUDA(cudaMemcpyAsync(m, w.ck.p + (long)(j0 / c->ckpt) * N, N * sizeof(T), cudaMemcpyDeviceToDevice,
                               c->s));
      for (int j = j0; j < j1; ++j) {
        const T* vA = vel_node<T>(c, vcoef, j, va);
        const T* wA = vel_node<T>(c, wcoef, j, wa);
        fused::AdvEpi<T> sA = adv_epi<T>(c, vA, m, yhS, accS, 1, nullptr, wA, sj);
        if (j == 0) {
          // the state's stage 1 leaves the spectrum of yhS for its stage 2
          adv<T>(c, m, vA, nullptr, nullptr, m, yhS, accS, nullptr, 1, nullptr, wA, sj, false, true, true);
        } else {
          fused::AdvEpi<T> iB = adv_epi<T>(c, vA, acc, y, nullptr, 2);
          iB.src_from_a = 1;
          adv2<T>(c, m, sA, yh, iB);
          if (mtil)
            REG_CUDA(cudaMemcpyAsync(mtil + (long)j * N, y, N * sizeof(T), cudaMemcpyDeviceToDevice, c->s));
        }
        const T* vB = vel_node<T>(c, vcoef, j + 1, vb);
        if (j == 0) {
          adv<T>(c, yhS, vB, nullptr, nullptr, accS, m, nullptr, nullptr, 2, nullptr, nullptr, nullptr, true);
          lincomb_t<T>(-h, sj, (T)0, nullptr, yh, N, c->s);
          lincomb_t<T>((T)(-0.5) * h, sj, (T)0, nullptr, acc, N, c->s);
        } else {
          fused::AdvEpi<T> sB = adv_epi<T>(c, vB, accS, m, nullptr, 2);
          fused::AdvEpi<T> iA = adv_epi<T>(c, vA, y, yh, acc, 1, sj);
          adv2<T>(c, yhS, sB, y, iA);
        }
      }
    }
    // the source at t_{n_t} from the final state, and the last incremental stage 2
    const T* vN = vel_node<T>(c, vcoef, c->n_t, va);
    fused::AdvEpi<T> sN = adv_epi<T>(c, nullptr, nullptr, nullptr, nullptr, 1, nullptr,
                                     vel_node<T>(c, wcoef, c->n_t, wa), sj);
    fused::AdvEpi<T> iN = adv_epi<T>(c, vN, acc, y, nullptr, 2);
    iN.src_from_a = 1;
    adv2<T>(c, m, sN, yh, iN);
    if (mtil)
      REG_CUDA(cudaMemcpyAsync(mtil + (long)c->n_t * N, y, N * sizeof(T), cudaMemcpyDeviceToDevice, c->s));
  }
  // each stage leaves the spectrum of its out1 in w.U for the next one (the
  // state re-advance of a segment overwrites it); the predictor yh is needed
  // only as that spectrum
  bool ready = false;
  for (int seg = 0; seg * K < c->n_t && !(use_src && c->ckpt > 0 && c->d == 3); ++seg) {
    int j0 = seg * K, j1 = j0 + K;
    int base = 0;
    if (c->ckpt > 0) {
      if (use_src) recompute_segment_src<T>(c, vcoef, wcoef, j0, j1);
      else recompute_segment<T>(c, vcoef, j0, j1);
      base = j0;
      ready = false;
    }
    for (int j = j0; j < j1; ++j) {
      const T* vA = vel_node<T>(c, vcoef, j, va);
      const bool more = j + 1 < j1;  // the next stage of this segment reads the spectrum of y
      const bool yh_ready = j > 0;
      if (use_src) {
        const T* s1 = w.src.p + (long)(j - base) * N;
        const T* s2 = w.src.p + (long)(j + 1 - base) * N;
        if (j == 0) {  // zero state: k1 = -s_0
          lincomb_t<T>(-h, s1, (T)0, nullptr, yh, N, c->s);
          lincomb_t<T>((T)(-0.5) * h, s1, (T)0, nullptr, acc, N, c->s);
        } else {
          adv<T>(c, y, vA, nullptr, nullptr, y, yh, acc, nullptr, 1, s1, nullptr, nullptr, ready, true, true);
        }
        adv<T>(c, yh, vel_node<T>(c, vcoef, j + 1, vb), nullptr, nullptr, acc, y, nullptr, nullptr, 2, s2, nullptr,
               nullptr, yh_ready, more);
        if (mtil)
          REG_CUDA(cudaMemcpyAsync(mtil + (long)(j + 1) * N, y, N * sizeof(T), cudaMemcpyDeviceToDevice, c->s));
      } else {
        const T* g1 = gm_slot<T>(c, j, base);
        const T* g2 = gmh_slot<T>(c, j + 1, base);
        const T* wA = vel_node<T>(c, wcoef, j, wa);
        if (j == 0) {
          transport_stage1<T>(nullptr, vA, g1, wA, nullptr, h, yh, acc, c->d, N, c->s);
        } else {
          adv<T>(c, y, vA, g1, wA, y, yh, acc, nullptr, 1, nullptr, nullptr, nullptr, ready, true, true);
        }
        adv<T>(c, yh, vel_node<T>(c, vcoef, j + 1, vb), g2, vel_node<T>(c, wcoef, j + 1, wb), acc, y, nullptr,
               nullptr, 2, nullptr, nullptr, nullptr, yh_ready, more);
      }
      ready = more;
    }
  }
  // lam~_1 = -m~_1
  lincomb_t<T>((T)-1, y, (T)0, nullptr, y, N, c->s);
  if (c->hess == REG_HESS_NEWTON) newton_adjoint<T>(c, vcoef, wcoef, f);
  else adjoint_solve<T>(c, vcoef, f);
}

}  // namespace

namespace {

// ---------------------------------------------------------------------------
// Fourier-diagonal tail (FP64): out = beta (C (x) A) V + K^gamma F
// (App. A Eq. control-equation-expansion; Eq. eliminated-control). F may be null.
// ---------------------------------------------------------------------------
// Without the Leray projection the body force passes the tail unchanged, so it
// is added in physical space and only V is transformed.
void tail(reg_ctx* c, const double* V, const double* F, double* out) {
  const long Nc = c->g.Nc, N = c->N();
  const int ncd = c->n_c * c->d;
  double2* SV = c->SV.get((size_t)ncd * Nc);
  double2* SF = c->SF.get((size_t)ncd * Nc);
  Spectral<double>& sp = *c->sp64;
  const bool fspec = F && c->stokes;
  for (int q = 0; q < ncd; ++q) {
    sp.fwd(V + q * N, SV + q * Nc);
    if (fspec) sp.fwd(F + q * N, SF + q * Nc);
  }
  spec_tail(c->g, c->s, SV, fspec ? SF : nullptr, SF, c->n_c, c->beta, c->Cg_dev.p, c->rtype, c->stokes,
            c->g.B > 1 ? c->betas_dev.p : nullptr);
  for (int q = 0; q < ncd; ++q) sp.inv(SF + q * Nc, out + q * N);
  if (F && !fspec) lincomb_t<double>(1.0, out, 1.0, F, out, (long)ncd * N, c->s);
}

void precond(reg_ctx* c, const double* r, double* z) {
  const long Nc = c->g.Nc, N = c->N();
  const int ncd = c->n_c * c->d;
  double2* SV = c->SV.get((size_t)ncd * Nc);
  double2* SF = c->SF.get((size_t)ncd * Nc);
  Spectral<double>& sp = *c->sp64;
  for (int q = 0; q < ncd; ++q) sp.fwd(r + q * N, SV + q * Nc);
  spec_precond(c->g, c->s, SV, SF, c->n_c, c->beta, c->Ci_dev.p, c->rtype, c->g.B > 1 ? c->betas_dev.p : nullptr);
  for (int q = 0; q < ncd; ++q) sp.inv(SF + q * Nc, z + q * N);
}

double* red(reg_ctx* c) { return c->red.get(reduce_scratch_doubles()); }

// beta/2 sum_ll' c_ll' <B v_l, B v_l'>_h
double reg_term(reg_ctx* c, const double* v) {
  double* Rv = c->tmpB.get(c->ncdN());
  tail(c, v, nullptr, Rv);
  return 0.5 * c->hd * dot(v, Rv, c->ncdN(), red(c), c->s);
}

void objective(reg_ctx* c, const double* v, double parts[2]) {
  if (!c->have_images) throw StatusError{REG_EINVAL, "reg_set_images has not been called"};
  const long N = c->N();
  Work<double>& w = c->w64;
  REG_CUDA(cudaMemcpyAsync(w.m.get(N), c->mT.p, N * sizeof(double), cudaMemcpyDeviceToDevice, c->s));
  state_steps<double>(c, v, 0, c->n_t, nullptr, nullptr, 0, nullptr);
  parts[0] = 0.5 * c->hd * sqdiff(c->mR.p, w.m.p, N, red(c), c->s);
  parts[1] = reg_term(c, v);
}

// FP32 copies of the stored state for the mixed-precision matvec
void prepare_mixed(reg_ctx* c) {
  if (c->prec != REG_MIXED) return;
  Work<double>& w = c->w64;
  Work<float>& x = c->w32;
  const long dN = c->dN(), N = c->N();
  spectral<float>(c);
  convert<double, float>(c->vlin.p, x.vcoef.get(c->ncdN()), c->ncdN(), c->s);
  if (c->hess == REG_HESS_NEWTON) {
    convert<double, float>(w.m1.p, x.m1.get(N), N, c->s);
    convert<double, float>(w.mR.p, x.mR.get(N), N, c->s);
  }
  if (c->ckpt == 0) {
    convert<double, float>(w.gm.p, x.gm.get((size_t)(c->n_t + 1) * dN), (long)(c->n_t + 1) * dN, c->s);
    if (c->quad) convert<double, float>(w.gmh.p, x.gmh.get((size_t)(c->n_t + 1) * dN), (long)(c->n_t + 1) * dN, c->s);
  } else {
    long nck = c->n_t / c->ckpt + 1;
    convert<double, float>(w.ck.p, x.ck.get((size_t)nck * N), nck * N, c->s);
  }
}

void set_point(reg_ctx* c, const double* v) {
  if (!c->have_images) throw StatusError{REG_EINVAL, "reg_set_images has not been called"};
  c->ready = false;
  REG_CUDA(cudaMemcpyAsync(c->vlin.get(c->ncdN()), v, c->ncdN() * sizeof(double), cudaMemcpyDeviceToDevice, c->s));
  state_solve_store<double>(c, c->vlin.p, c->mT.p);
  if (c->hess == REG_HESS_NEWTON) {  // m_1 and m_R for the adjoint inside the Newton matvec
    const long N = c->N();
    REG_CUDA(cudaMemcpyAsync(c->w64.m1.get(N), c->w64.m.p, N * sizeof(double), cudaMemcpyDeviceToDevice, c->s));
    REG_CUDA(cudaMemcpyAsync(c->w64.mR.get(N), c->mR.p, N * sizeof(double), cudaMemcpyDeviceToDevice, c->s));
  }
}

void check_finite(double x, const char* what) {
  if (!std::isfinite(x)) throw StatusError{REG_ENONFINITE, std::string(what) + " is not finite"};
}

// gradient at v; parts = {distance, regularisation}
void gradient(reg_ctx* c, const double* v, double* g, double parts[2]) {
  const long N = c->N();
  set_point(c, v);
  Work<double>& w = c->w64;
  // w.m holds m_1 after the state solve
  parts[0] = 0.5 * c->hd * sqdiff(c->mR.p, w.m.p, N, red(c), c->s);
  lincomb_t<double>(1.0, c->mR.p, -1.0, w.m.p, w.lam.get(N), N, c->s);  // lam_1 = m_R - m_1
  double* f = c->f.get(c->ncdN());
  adjoint_solve<double>(c, c->vlin.p, f);
  tail(c, c->vlin.p, f, g);
  parts[1] = reg_term(c, c->vlin.p);
  check_finite(parts[0] + parts[1], "objective");
  check_finite(dot(g, g, c->ncdN(), red(c), c->s), "gradient norm");
  prepare_mixed(c);
  c->ready = true;
}

void hessvec_body(reg_ctx* c, const double* vt, double* out) {
  double* f = c->f.get(c->ncdN());
  if (c->prec == REG_FP64) {
    gn_sweeps<double>(c, c->vlin.p, vt, f);
  } else {
    float* w32 = c->w32.wcoef.get(c->ncdN());
    convert<double, float>(vt, w32, c->ncdN(), c->s);
    gn_sweeps<float>(c, c->w32.vcoef.p, w32, f);
  }
  tail(c, vt, f, out);
}

// addresses of every buffer the captured matvec touches: a change means the
// graph would read or write stale memory and must be captured again
size_t graph_signature(reg_ctx* c) {
  const void* ptrs[] = {c->f.p,        c->SV.p,       c->SF.p,       c->vlin.p,     c->gdir.p,     c->gout.p,
                        c->w64.U.p,    c->w64.W.p,    c->w64.X.p,    c->w64.m.p,    c->w64.yh.p,   c->w64.acc.p,
                        c->w64.lam.p,  c->w64.va.p,   c->w64.vb.p,   c->w64.wa.p,   c->w64.wb.p,   c->w64.gm.p,
                        c->w64.gmh.p,  c->w64.ck.p,   c->w32.U.p,    c->w32.W.p,    c->w32.X.p,    c->w32.m.p,
                        c->w32.yh.p,   c->w32.acc.p,  c->w32.lam.p,  c->w32.va.p,   c->w32.vb.p,   c->w32.wa.p,
                        c->w32.wb.p,   c->w32.gm.p,   c->w32.gmh.p,  c->w32.ck.p,   c->w32.vcoef.p, c->w32.wcoef.p,
                        c->w32.fhi.p,  c->w32.flo.p,  c->w64.G.p,    c->w32.G.p,    c->w64.src.p,  c->w32.src.p,
                        c->w64.mtil.p, c->w32.mtil.p, c->w64.lamN.p, c->w32.lamN.p, c->w64.yh2.p, c->w32.yh2.p,
                        c->w64.acc2.p, c->w32.acc2.p, c->w64.st0.p,  c->w32.st0.p,  c->w64.st1.p,  c->w32.st1.p,
                        c->w64.Gt.p,   c->w32.Gt.p,   c->w64.U2.p,   c->w32.U2.p,   c->w64.W2.p,   c->w32.W2.p,
                        c->w64.X2.p,   c->w32.X2.p,   c->w64.yhS.p,  c->w32.yhS.p,  c->w64.accS.p, c->w32.accS.p,
                        c->w64.srcS.p, c->w32.srcS.p};
  size_t h = 1469598103934665603ull;
  for (const void* p : ptrs) h = (h ^ (size_t)p) * 1099511628211ull;
  // and the settings that change what the matvec computes
  uint64_t bb;
  std::memcpy(&bb, &c->beta, sizeof bb);
  const uint64_t modes[] = {bb, (uint64_t)c->hess, (uint64_t)c->quad, (uint64_t)c->prec, (uint64_t)c->n_t};
  for (uint64_t m : modes) h = (h ^ (size_t)m) * 1099511628211ull;
  return h;
}

void hessvec(reg_ctx* c, const double* vt, double* out) {
  if (!c->ready) throw StatusError{REG_ENOTREADY, "no linearisation point: call reg_gradient or reg_linearize first"};
  if (!c->graphs || !c->s || c->prof.mask) {
    hessvec_body(c, vt, out);
    return;
  }
  const long n = c->ncdN();
  double* gvt = c->gdir.get(n);
  double* gout = c->gout.get(n);
  if (!c->gexec || graph_signature(c) != c->gsig) {
    if (c->gexec) {
      cudaGraphExecDestroy(c->gexec);
      c->gexec = nullptr;
    }
    // one ordinary run allocates every buffer (and tunes the passes) first
    REG_CUDA(cudaMemcpyAsync(gvt, vt, n * sizeof(double), cudaMemcpyDeviceToDevice, c->s));
    hessvec_body(c, gvt, gout);
    REG_CUDA(cudaStreamSynchronize(c->s));
    long l0 = launch_count();
    cudaGraph_t graph = nullptr;
    REG_CUDA(cudaStreamBeginCapture(c->s, cudaStreamCaptureModeThreadLocal));
    try {
      hessvec_body(c, gvt, gout);
    } catch (...) {
      cudaStreamEndCapture(c->s, &graph);
      if (graph) cudaGraphDestroy(graph);
      throw;
    }
    REG_CUDA(cudaStreamEndCapture(c->s, &graph));
    cudaError_t e = cudaGraphInstantiate(&c->gexec, graph, 0);
    cudaGraphDestroy(graph);
    REG_CUDA(e);
    c->gkernels = launch_count() - l0;
    c->gsig = graph_signature(c);
  }
  REG_CUDA(cudaMemcpyAsync(gvt, vt, n * sizeof(double), cudaMemcpyDeviceToDevice, c->s));
  REG_CUDA(cudaGraphLaunch(c->gexec, c->s));
  add_launches(c->gkernels);
  REG_CUDA(cudaMemcpyAsync(out, gout, n * sizeof(double), cudaMemcpyDeviceToDevice, c->s));
}

Coefs basis_at(const reg_ctx* c, double t) {
  Coefs b{};
  cheb_values(c->n_c, t, b.c);
  return b;
}

double cfl(reg_ctx* c, const double* v) {
  const long N = c->N(), dN = c->dN();
  double* vt = c->tmpA.get(dN);
  double mx = 0.0;
  int nodes = c->n_c == 1 ? 1 : c->n_t + 1;
  for (int j = 0; j < nodes; ++j) {
    const double* vj = v;
    if (c->n_c > 1) {
      vel_at<double, double>(v, c->n_c, c->basis_at_node(j), vt, dN, c->s);
      vj = vt;
    }
    for (int i = 0; i < c->d; ++i) {
      double hx = 2.0 * M_PI / c->g.n[i];
      mx = std::max(mx, maxabs(vj + i * N, N, red(c), c->s) / hx);
    }
  }
  return c->h() * mx;
}

// F_1 (App. D Eq. def-grad) with substeps * n_t Heun steps; returns c->F
double* defgrad(reg_ctx* c, const double* v, int substeps) {
  const long N = c->N(), dN = c->dN();
  const int d = c->d, dd = d * d, nc = c->n_c;
  const long ddN = (long)dd * N;
  double* gvl = c->gvl.get((size_t)nc * ddN);
  for (int l = 0; l < nc; ++l)
    for (int i = 0; i < d; ++i) grad_into<double>(c, v + ((long)l * d + i) * N, gvl + ((long)l * dd + i * d) * N);
  double* F = c->F.get(ddN);
  double* Fh = c->Fh.get(ddN);
  double* K1 = c->K1.get(ddN);
  double* K2 = c->K2.get(ddN);
  double* gvt = c->gvt.get(ddN);
  double* vt = c->tmpA.get(dN);
  double* G = c->w64.G.get(dN);
  identity_tensor(F, d, N, c->s);
  const int nF = c->n_t * substeps;
  const double h = 1.0 / nF;
  for (int j = 0; j < nF; ++j) {
    for (int stage = 0; stage < 2; ++stage) {
      double t = (double)(j + stage) * h;
      const double* vv = v;
      const double* gg = gvl;
      if (nc > 1) {
        Coefs b = basis_at(c, t);
        vel_at<double, double>(v, nc, b, vt, dN, c->s);
        vel_at<double, double>(gvl, nc, b, gvt, ddN, c->s);
        vv = vt;
        gg = gvt;
      }
      const double* Fin = stage ? Fh : F;
      double* Kout = stage ? K2 : K1;
      for (int q = 0; q < dd; ++q) {
        grad_into<double>(c, Fin + q * N, G);
        detF_rhs(G, vv, gg, Fin, q, Kout, d, N, c->s);
      }
      if (stage == 0) {
        lincomb(1.0, F, h, K1, Fh, ddN, c->s);
      } else {
        axpby(0.5 * h, K1, 1.0, F, ddN, c->s);
        axpby(0.5 * h, K2, 1.0, F, ddN, c->s);
      }
    }
  }
  return F;
}

// det F_1 statistics {min, max, mean, std} (and the field, if det_out)
void detF(reg_ctx* c, const double* v, int substeps, double st[4], double* det_out) {
  const long N = c->N();
  double* F = defgrad(c, v, substeps);
  double* det = det_out ? det_out : c->det.get(N);
  det_tensor(F, det, c->d, N, c->s);
  stats(det, N, red(c), c->s, st);
}

reg_ctx* create_ctx(int d, const int64_t* n, int n_t, int n_c, double beta, int reg_type, int stokes, int precision,
                    int ckpt_every, void* cuda_stream, int batch);

// det F_1 statistics on a grid refined `refine` times per axis: the velocity,
// band-limited on the context's grid, is carried to the finer grid exactly by
// trigonometric interpolation (its spectrum padded with zeros), and Eq.
// def-grad is integrated there, where the products of the F-equation are
// resolved. det_out (may be null): the N * refine^d values of the fine grid.
void detF_refined(reg_ctx* c, const double* v, int substeps, int refine, double st[4], double* det_out) {
  if (refine == 1) return detF(c, v, substeps, st, det_out);
  if (c->g.B > 1) throw StatusError{REG_EINVAL, "refined det F needs a single problem"};
  int64_t nf[3] = {1, 1, 1};
  for (int a = 0; a < c->d; ++a) {
    nf[a] = (int64_t)c->g.n[a] * refine;
    if (nf[a] > 512) throw StatusError{REG_EINVAL, "refined grid exceeds 512 points per axis"};
  }
  std::unique_ptr<reg_ctx> f(create_ctx(c->d, nf, c->n_t, c->n_c, c->beta, c->rtype, c->stokes, REG_FP64, 0, c->s, 1));
  const int ncd = c->n_c * c->d;
  const long N = c->N(), Nc = c->g.Nc;
  double2* P = c->SV.get((size_t)ncd * Nc);
  for (int q = 0; q < ncd; ++q) c->sp64->fwd(v + q * N, P + q * Nc);
  double2* Q = f->SV.get((size_t)ncd * f->g.Nc);
  spec_upsample(c->g, f->g, c->s, P, Q, ncd);
  double* vf = f->vlin.get(f->ncdN());
  for (int q = 0; q < ncd; ++q) f->sp64->inv(Q + q * f->g.Nc, vf + q * f->N());
  detF(f.get(), vf, substeps, st, det_out);
  REG_CUDA(cudaStreamSynchronize(c->s));  // the fine context's buffers are freed on return
}

// det F_1 and grid-angle statistics from one F_1 (either field output may be null)
void deform_measures(reg_ctx* c, const double* v, int substeps, double det_st[4], double ang_st[4], double* det_out,
                     double* ang_out) {
  const long N = c->N();
  double* F = defgrad(c, v, substeps);
  double* det = det_out ? det_out : c->det.get(N);
  det_tensor(F, det, c->d, N, c->s);
  stats(det, N, red(c), c->s, det_st);
  double* ang = ang_out ? ang_out : c->ang.get(N);
  grid_angle_tensor(F, ang, c->d, N, c->s);
  stats(ang, N, red(c), c->s, ang_st);
}

// Gaussian presmoothing of one FP64 field (Sec. 3.3.5 "Presmoothing")
void smooth(reg_ctx* c, double sigma, const double* in, double* out) {
  const long Nc = c->g.Nc;
  double2* S = c->SV.get((size_t)c->n_c * c->d * Nc);
  double2* T = c->SF.get((size_t)c->n_c * c->d * Nc);
  c->sp64->fwd(in, S);
  spec_gauss(c->g, c->s, S, T, sigma);
  c->sp64->inv(T, out);
}

// Deformation map (App. D Eq. displacement): du_i/dt = -v . grad u_i + v_i,
// u_0 = 0, the same fused Heun stages as the state equation with the source
// -v_i(t) (the stage subtracts its source). u: d fields.
void displacement(reg_ctx* c, const double* v, double* u) {
  Work<double>& w = c->w64;
  const long N = c->N(), dN = c->dN();
  double* yh = w.yh.get(N);
  double* acc = w.acc.get(N);
  double* va = w.va.get(dN);
  double* vb = w.vb.get(dN);
  double* s1 = c->disp_src.get(2 * N);
  double* s2 = s1 + N;
  REG_CUDA(cudaMemsetAsync(u, 0, dN * sizeof(double), c->s));
  for (int j = 0; j < c->n_t; ++j) {
    const double* vA = vel_node<double>(c, v, j, va);
    const double* vB = vel_node<double>(c, v, j + 1, vb);
    for (int i = 0; i < c->d; ++i) {
      double* ui = u + (long)i * N;
      lincomb_t<double>(-1.0, vA + (long)i * N, 0.0, nullptr, s1, N, c->s);
      lincomb_t<double>(-1.0, vB + (long)i * N, 0.0, nullptr, s2, N, c->s);
      adv<double>(c, ui, vA, nullptr, nullptr, ui, yh, acc, nullptr, 1, s1);
      adv<double>(c, yh, vB, nullptr, nullptr, acc, ui, nullptr, nullptr, 2, s2);
    }
  }
}

// Eigenvalues of the symmetric tridiagonal matrix with diagonal a[0..m) and
// off-diagonal b[0..m-1), ascending: bisection on Sturm counts (the number of
// negative pivots of T - x I; Golub & Van Loan Sec. 8.4.1) inside the
// Gershgorin interval.
void tridiag_eigs(const double* a, const double* b, int m, double* out) {
  double lo = a[0], hi = a[0];
  for (int i = 0; i < m; ++i) {
    double r = (i > 0 ? std::fabs(b[i - 1]) : 0.0) + (i + 1 < m ? std::fabs(b[i]) : 0.0);
    lo = std::min(lo, a[i] - r);
    hi = std::max(hi, a[i] + r);
  }
  const double scale = std::max(std::fabs(lo), std::fabs(hi));
  const double tiny = DBL_MIN / DBL_EPSILON;
  auto count_below = [&](double x) {
    int cnt = 0;
    double dd = a[0] - x;
    if (dd < 0) ++cnt;
    for (int i = 1; i < m; ++i) {
      if (std::fabs(dd) < tiny) dd = dd < 0 ? -tiny : tiny;
      dd = a[i] - x - b[i - 1] * b[i - 1] / dd;
      if (dd < 0) ++cnt;
    }
    return cnt;
  };
  for (int k = 0; k < m; ++k) {  // the k-th smallest eigenvalue lies where the count passes k
    double l = lo, h = hi;
    for (int it = 0; it < 200 && h - l > 2.0 * DBL_EPSILON * scale; ++it) {
      double mid = 0.5 * (l + h);
      if (count_below(mid) > k) h = mid;
      else l = mid;
    }
    out[k] = 0.5 * (l + h);
  }
}

// Lanczos three-term recurrence (Sec. 3.3.5 "Regularization"; Golub & Van
// Loan Sec. 9.1) on the Hessian at the linearisation point, or on P^{-1} H in
// the P inner product. Returns the number of steps completed.
int lanczos(reg_ctx* c, const double* q0, int k, int use_precond, double* alpha, double* beta) {
  const long n = c->ncdN();
  double* q = c->lz_q.get(n);
  double* u = c->lz_u.get(n);
  double* up = c->lz_up.get(n);
  double* w = c->lz_w.get(n);
  double* z = c->lz_z.get(n);
  double* rs = red(c);
  REG_CUDA(cudaMemcpyAsync(u, q0, n * sizeof(double), cudaMemcpyDeviceToDevice, c->s));
  if (use_precond) precond(c, u, q);
  else REG_CUDA(cudaMemcpyAsync(q, u, n * sizeof(double), cudaMemcpyDeviceToDevice, c->s));
  double nrm2 = dot(u, q, n, rs, c->s);
  if (!(nrm2 > 0.0) || !std::isfinite(nrm2)) throw StatusError{REG_EINVAL, "the start vector has no positive norm"};
  double nrm = std::sqrt(nrm2);
  axpby(0.0, q, 1.0 / nrm, q, n, c->s);
  axpby(0.0, u, 1.0 / nrm, u, n, c->s);
  REG_CUDA(cudaMemsetAsync(up, 0, n * sizeof(double), c->s));
  double bprev = 0.0;
  int steps = 0;
  for (int j = 0; j < k; ++j) {
    hessvec(c, q, w);
    axpby(-bprev, up, 1.0, w, n, c->s);
    double a = dot(q, w, n, rs, c->s);
    axpby(-a, u, 1.0, w, n, c->s);
    if (use_precond) precond(c, w, z);
    else REG_CUDA(cudaMemcpyAsync(z, w, n * sizeof(double), cudaMemcpyDeviceToDevice, c->s));
    double b2 = dot(w, z, n, rs, c->s);
    check_finite(a, "Lanczos alpha");
    check_finite(b2, "Lanczos beta");
    double b = b2 > 0.0 ? std::sqrt(b2) : 0.0;
    alpha[j] = a;
    beta[j] = b;
    steps = j + 1;
    if (b == 0.0) break;
    std::swap(up, u);  // u_{j-1} <- u_j, then u_{j+1} = w / b
    lincomb(1.0 / b, w, 0.0, w, u, n, c->s);
    lincomb(1.0 / b, z, 0.0, z, q, n, c->s);
    bprev = b;
  }
  return steps;
}

// Time steps of the context (n_t) changed: node basis values, stored state invalid
void set_time_steps(reg_ctx* c, int n_t) {
  if (n_t < 1) throw StatusError{REG_EINVAL, "n_t must be >= 1"};
  if (c->ckpt > 0 && n_t % c->ckpt != 0) throw StatusError{REG_EINVAL, "n_t must be a multiple of ckpt_every"};
  c->n_t = n_t;
  c->bnode.assign((size_t)(n_t + 1) * c->n_c, 0.0);
  for (int j = 0; j <= n_t; ++j) cheb_values(c->n_c, (double)j / n_t, &c->bnode[(size_t)j * c->n_c]);
  c->ready = false;
}

// ---------------------------------------------------------------------------
// Termination test at iterate k: the relative gradient reduction, or the set
// C1-C5 of Eq. stopping-criteria combined as in Eq. converged. Returns true to
// stop; maxed is set when only the iteration cap stops the solve.
// ---------------------------------------------------------------------------
bool stop_test(const reg_solve_opts& o, reg_solve_report& R, int k, double ginf, bool& maxed) {
  maxed = false;
  R.stop_flags = 0;
  if (o.stop_rule == REG_STOP_GRAD_REL) {
    if (ginf <= o.grad_rtol * R.g0_inf) return true;
    maxed = k >= o.max_outer;
    return maxed;
  }
  const double tau = o.tau_J, one_J0 = 1.0 + R.J0;
  int f = 0;
  if (k >= 1 && R.J_prev - R.J < tau * one_J0) f |= 1;             // C1
  if (k >= 1 && R.dv_inf < std::sqrt(tau) * (1.0 + R.v_inf)) f |= 2; // C2
  if (ginf < std::cbrt(tau) * one_J0) f |= 4;                       // C3
  if (ginf < 1e3 * DBL_EPSILON) f |= 8;                             // C4
  if (k > o.max_outer) f |= 16;                                     // C5
  R.stop_flags = f;
  if ((f & 7) == 7 || (f & 8)) return true;
  maxed = (f & 16) != 0;
  return maxed;
}

// ---------------------------------------------------------------------------
// Alg. 1: the outer loop. Search direction: the inexact (Gauss-)Newton step
// from PCG (Nocedal & Wright Alg. 5.3) with the forcing term of Eq.
// termination-criterion-ksm, or the Picard update -P^{-1} g (Eq. picard,
// App. C) scaled by the step memory alpha~; then CFL halving and Armijo
// backtracking.
// ---------------------------------------------------------------------------
int solve(reg_ctx* c, double* v, const reg_solve_opts& o, reg_solve_report& R) {
  auto t0 = std::chrono::steady_clock::now();
  if (o.method != REG_METHOD_KRYLOV && o.method != REG_METHOD_PICARD) throw StatusError{REG_EINVAL, "bad method"};
  if (o.stop_rule != REG_STOP_GRAD_REL && o.stop_rule != REG_STOP_C1C5) throw StatusError{REG_EINVAL, "bad stop_rule"};
  if (o.stop_rule == REG_STOP_C1C5 && !(o.tau_J > 0.0)) throw StatusError{REG_EINVAL, "tau_J must be positive"};
  const long n = c->ncdN();
  double* g = c->sv_g.get(n);
  double* s = c->sv_s.get(n);
  double* r = c->sv_r.get(n);
  double* z = c->sv_z.get(n);
  double* p = c->sv_p.get(n);
  double* Hp = c->sv_Hp.get(n);
  double* vt = c->sv_vt.get(n);
  double* rs = red(c);
  std::memset(&R, 0, sizeof(R));
  double parts[2];
  gradient(c, v, g, parts);
  R.n_pde += 2;
  double J = parts[0] + parts[1];
  R.J0 = J;
  R.g0_inf = maxabs(g, n, rs, c->s);
  R.v_inf = maxabs(v, n, rs, c->s);
  double amem = 1.0;
  R.alpha_mem = amem;
  double g0_2 = std::sqrt(dot(g, g, n, rs, c->s));
  long maxit = o.pcg_maxit > 0 ? o.pcg_maxit : n;
  int status = REG_OK;
  int k = 0;
  for (;;) {
    double ginf = maxabs(g, n, rs, c->s);
    double g2 = std::sqrt(dot(g, g, n, rs, c->s));
    R.g_inf = ginf;
    R.J = J;
    bool maxed = false;
    if (stop_test(o, R, k, ginf, maxed)) {
      if (maxed) status = REG_EMAXIT;
      break;
    }
    if (o.method == REG_METHOD_PICARD) {
      precond(c, g, s);
      axpby(0.0, s, o.step_memory ? -amem : -1.0, s, n, c->s);
    } else {
      double eta = std::min(0.5, std::sqrt(g2 / g0_2));
      // PCG on H s = -g from s = 0
      REG_CUDA(cudaMemsetAsync(s, 0, n * sizeof(double), c->s));
      REG_CUDA(cudaMemcpyAsync(r, g, n * sizeof(double), cudaMemcpyDeviceToDevice, c->s));
      precond(c, r, z);
      lincomb(-1.0, z, 0.0, z, p, n, c->s);
      double rz = dot(r, z, n, rs, c->s);
      for (long it = 0; it < maxit; ++it) {
        double rn = std::sqrt(dot(r, r, n, rs, c->s));
        check_finite(rn, "PCG residual");
        if (rn <= eta * g2) break;
        hessvec(c, p, Hp);
        R.matvecs += 1;
        R.n_pde += 2;
        R.pcg_iters += 1;
        double pHp = dot(p, Hp, n, rs, c->s);
        check_finite(pHp, "PCG curvature");
        if (pHp <= 0.0) {
          if (it == 0) REG_CUDA(cudaMemcpyAsync(s, p, n * sizeof(double), cudaMemcpyDeviceToDevice, c->s));
          break;
        }
        double alpha = rz / pHp;
        axpby(alpha, p, 1.0, s, n, c->s);
        axpby(alpha, Hp, 1.0, r, n, c->s);
        precond(c, r, z);
        double rz_new = dot(r, z, n, rs, c->s);
        double bta = rz_new / rz;
        rz = rz_new;
        axpby(-1.0, z, bta, p, n, c->s);
      }
    }
    // keep the step inside the CFL bound by halving it (Sec. 3.3.5)
    if (o.cfl_max > 0) {
      int halvings = 0;
      for (;;) {
        lincomb(1.0, v, 1.0, s, vt, n, c->s);
        if (cfl(c, vt) <= o.cfl_max) break;
        if (++halvings > 30) throw StatusError{REG_ECFL, "CFL bound not met after 30 step halvings"};
        axpby(0.0, s, 0.5, s, n, c->s);
        R.cfl_halvings += 1;
      }
    }
    // Armijo backtracking from alpha = 1
    double slope = c->hd * dot(g, s, n, rs, c->s);
    double alpha = 1.0, Jt = 0.0;
    bool accepted = false;
    for (int t = 0; t < o.max_backtracks; ++t) {
      lincomb(1.0, v, alpha, s, vt, n, c->s);
      double pt[2];
      objective(c, vt, pt);
      R.ls_trials += 1;
      R.n_pde += 1;
      Jt = pt[0] + pt[1];
      if (std::isfinite(Jt) && Jt <= J + o.armijo_c1 * alpha * slope) {
        accepted = true;
        break;
      }
      alpha *= o.backtrack;
    }
    if (!accepted) {
      status = REG_ELINESEARCH;
      break;
    }
    // step memory: doubled after a full step, else scaled by the accepted alpha
    if (o.method == REG_METHOD_PICARD && o.step_memory) amem = (alpha == 1.0) ? 2.0 * amem : amem * alpha;
    R.alpha_mem = amem;
    lincomb(1.0, vt, -1.0, v, r, n, c->s);  // v_k - v_{k-1}
    R.dv_inf = maxabs(r, n, rs, c->s);
    REG_CUDA(cudaMemcpyAsync(v, vt, n * sizeof(double), cudaMemcpyDeviceToDevice, c->s));
    R.v_inf = maxabs(v, n, rs, c->s);
    R.J_prev = J;
    gradient(c, v, g, parts);
    R.n_pde += 2;
    J = parts[0] + parts[1];
    k += 1;
  }
  R.outer = k;
  R.J = J;
  double base = sqdiff(c->mT.p, c->mR.p, c->N(), rs, c->s);
  double pt[2];
  objective(c, v, pt);
  R.dist_rel = base > 0 ? (2.0 * pt[0] / c->hd) / base : 0.0;
  R.cfl = cfl(c, v);
  if (o.detF_substeps > 0) detF_refined(c, v, o.detF_substeps, o.detF_refine > 1 ? o.detF_refine : 1, R.detF, nullptr);
  REG_CUDA(cudaStreamSynchronize(c->s));
  R.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  R.status = status;
  return status;
}

// ---------------------------------------------------------------------------
// Parameter continuation in beta (Sec. 3.3.5 "Regularization"): reduce beta
// by 10x from beta0 while the bounds on det F_1 (and the grid angle) hold,
// then bisect between the last accepted and the breaching beta.
// ---------------------------------------------------------------------------
int continuation(reg_ctx* c, double* v, const reg_solve_opts& so, const reg_cont_opts& co, reg_cont_report& R) {
  auto t0 = std::chrono::steady_clock::now();
  if (!(co.beta0 > 0.0) || !(co.beta_min > 0.0) || !(co.beta_rtol > 0.0) || !(co.dist_rtol >= 0.0) ||
      !(co.eps_F >= 0.0 && co.eps_F < 1.0) || !(co.eps_theta >= 0.0 && co.eps_theta < 0.5 * M_PI) ||
      co.detF_substeps < 1 || co.max_solves < 1 || !(co.cfl_target >= 0.0))
    throw StatusError{REG_EINVAL, "bad continuation options"};
  const long n = c->ncdN();
  double* vstart = c->ct_start.get(n);
  double* vgood = c->ct_good.get(n);
  REG_CUDA(cudaMemcpyAsync(vstart, v, n * sizeof(double), cudaMemcpyDeviceToDevice, c->s));
  std::memset(&R, 0, sizeof(R));
  bool have_good = false, bisect = false;
  double beta_good = 0.0, beta_bad = 0.0, dist_prev = -1.0;
  double beta = co.beta0;
  for (;;) {
    if (R.solves >= co.max_solves) {
      R.stop = 4;
      break;
    }
    c->beta = beta;
    REG_CUDA(cudaMemcpyAsync(v, have_good ? vgood : vstart, n * sizeof(double), cudaMemcpyDeviceToDevice, c->s));
    reg_solve_report sr;
    int st = solve(c, v, so, sr);
    R.solves += 1;
    R.outer += sr.outer;
    R.pcg_iters += sr.pcg_iters;
    R.matvecs += sr.matvecs;
    // a solve ended by the iteration cap or a failed line search keeps its last iterate
    if (st != REG_OK && st != REG_EMAXIT && st != REG_ELINESEARCH)
      throw StatusError{st, "a solve of the continuation failed"};
    if (co.cfl_target > 0.0 && sr.cfl > co.cfl_target) {
      // more time steps in proportion to the CFL excess, then the same beta again
      const int K = c->ckpt > 0 ? c->ckpt : 1;
      long want = (long)std::ceil(c->n_t * sr.cfl / co.cfl_target);
      want = (want + K - 1) / K * K;
      set_time_steps(c, (int)std::max<long>(want, c->n_t + K));
      continue;
    }
    double dst[4], ast[4];
    deform_measures(c, v, co.detF_substeps, dst, ast, nullptr, nullptr);
    const double dist = std::sqrt(sr.dist_rel);
    const bool ok = dst[0] >= co.eps_F && (co.eps_theta <= 0.0 || ast[0] >= co.eps_theta);
    if (R.n_trace < REG_CONT_TRACE) {
      int t = R.n_trace++;
      R.trace_beta[t] = beta;
      R.trace_detF[t] = dst[0];
      R.trace_angle[t] = ast[0];
      R.trace_dist[t] = dist;
      R.trace_ok[t] = ok;
    }
    if (ok) {
      have_good = true;
      beta_good = beta;
      REG_CUDA(cudaMemcpyAsync(vgood, v, n * sizeof(double), cudaMemcpyDeviceToDevice, c->s));
      R.detF_min = dst[0];
      R.angle_min = ast[0];
      R.dist_rel = sr.dist_rel;
    }
    if (!bisect) {
      if (ok) {
        if (dist_prev > 0.0 && dist_prev - dist < co.dist_rtol * dist_prev) {
          R.stop = 2;
          break;
        }
        dist_prev = dist;
        if (beta / 10.0 < co.beta_min) {
          R.stop = 1;
          break;
        }
        beta /= 10.0;
        continue;
      }
      R.beta_breach = beta;
      if (!have_good) {
        R.stop = 3;
        break;
      }
      beta_bad = beta;
      bisect = true;
    } else if (ok) {
      beta_good = beta;
    } else {
      beta_bad = beta;
    }
    const double next = 0.5 * (beta_good + beta_bad);
    if (std::fabs(next - beta) < co.beta_rtol * R.beta_breach) {
      R.stop = 0;
      break;
    }
    beta = next;
  }
  R.found = have_good;
  if (have_good) {
    REG_CUDA(cudaMemcpyAsync(v, vgood, n * sizeof(double), cudaMemcpyDeviceToDevice, c->s));
    c->beta = beta_good;
  }
  R.beta = c->beta;
  R.n_t = c->n_t;
  c->ready = false;
  REG_CUDA(cudaStreamSynchronize(c->s));
  R.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return REG_OK;
}

// ---------------------------------------------------------------------------
// Stacked problems (g.B > 1): per-problem objective and gradient, and the
// outer loop of Alg. 1 run for all problems in lockstep. Every kernel of a
// matvec, gradient or objective evaluation covers all problems at once; the
// Krylov and line-search scalars are per problem, so each problem follows
// exactly the iteration it would follow alone. A problem that has stopped
// keeps its iterate: its update coefficients are zero.
// ---------------------------------------------------------------------------
struct Seg {
  reg_ctx* c;
  int B, K;
  long N1;
  double* scr;
  std::vector<double> tmp;
  explicit Seg(reg_ctx* c_, int K_)
      : c(c_), B(c_->g.B), K(K_), N1(c_->g.N1), scr(c_->seg_scr.get(seg_scratch_doubles(c_->g.B))), tmp(c_->g.B) {}
  void dot(const double* a, const double* b, std::vector<double>& out) {
    out.resize(B);
    seg_dot(a, b, K, B, N1, scr, c->s, out.data());
  }
  void maxabs(const double* a, std::vector<double>& out) {
    out.resize(B);
    seg_maxabs(a, K, B, N1, scr, c->s, out.data());
  }
  // out = a_p x + b_p y (per-problem coefficients from the host)
  void comb(const std::vector<double>& a, const double* x, const std::vector<double>& b, const double* y, double* out) {
    double* da = c->coefA.get(B);
    double* db = c->coefC.get(B);
    REG_CUDA(cudaMemcpyAsync(da, a.data(), B * sizeof(double), cudaMemcpyHostToDevice, c->s));
    REG_CUDA(cudaMemcpyAsync(db, b.data(), B * sizeof(double), cudaMemcpyHostToDevice, c->s));
    REG_CUDA(cudaStreamSynchronize(c->s));  // the host vectors may change after return
    lincomb_seg(da, x, db, y, out, K, B, N1, c->s);
  }
};

// per problem: distance 1/2 h_d ||m_R - m_1||^2 and regularisation of v
void objective_seg(reg_ctx* c, const double* v, std::vector<double>& dist, std::vector<double>& regt) {
  const long N = c->N();
  Work<double>& w = c->w64;
  REG_CUDA(cudaMemcpyAsync(w.m.get(N), c->mT.p, N * sizeof(double), cudaMemcpyDeviceToDevice, c->s));
  state_steps<double>(c, v, 0, c->n_t, nullptr, nullptr, 0, nullptr);
  Seg one(c, 1), vec(c, c->n_c * c->d);
  dist.resize(c->g.B);
  seg_sqdiff(c->mR.p, w.m.p, 1, c->g.B, c->g.N1, one.scr, c->s, dist.data());
  for (double& x : dist) x *= 0.5 * c->hd;
  double* Rv = c->tmpB.get(c->ncdN());
  tail(c, v, nullptr, Rv);
  vec.dot(v, Rv, regt);
  for (double& x : regt) x *= 0.5 * c->hd;
}

void gradient_seg(reg_ctx* c, const double* v, double* g, std::vector<double>& dist, std::vector<double>& regt) {
  const long N = c->N();
  set_point(c, v);
  Work<double>& w = c->w64;
  Seg one(c, 1), vec(c, c->n_c * c->d);
  dist.resize(c->g.B);
  seg_sqdiff(c->mR.p, w.m.p, 1, c->g.B, c->g.N1, one.scr, c->s, dist.data());
  for (double& x : dist) x *= 0.5 * c->hd;
  lincomb_t<double>(1.0, c->mR.p, -1.0, w.m.p, w.lam.get(N), N, c->s);
  double* f = c->f.get(c->ncdN());
  adjoint_solve<double>(c, c->vlin.p, f);
  tail(c, c->vlin.p, f, g);
  double* Rv = c->tmpB.get(c->ncdN());
  tail(c, c->vlin.p, nullptr, Rv);
  vec.dot(c->vlin.p, Rv, regt);
  for (double& x : regt) x *= 0.5 * c->hd;
  prepare_mixed(c);
  c->ready = true;
}

// per-problem CFL number of coefficient vector v
void cfl_seg(reg_ctx* c, const double* v, std::vector<double>& out) {
  const int B = c->g.B;
  const long N1 = c->g.N1, N = c->N(), dN = c->dN();
  out.assign(B, 0.0);
  Seg one(c, 1);
  std::vector<double> m;
  double* vt = c->tmpA.get(dN);
  const int nodes = c->n_c == 1 ? 1 : c->n_t + 1;
  for (int j = 0; j < nodes; ++j) {
    const double* vj = v;
    if (c->n_c > 1) {
      vel_at<double, double>(v, c->n_c, c->basis_at_node(j), vt, dN, c->s);
      vj = vt;
    }
    for (int i = 0; i < c->d; ++i) {
      seg_maxabs(vj + (long)i * N, 1, B, N1, one.scr, c->s, (one.tmp.resize(B), one.tmp.data()));
      const double hx = 2.0 * M_PI / c->g.n[i];
      for (int p = 0; p < B; ++p) out[p] = std::max(out[p], c->h() * one.tmp[p] / hx);
    }
  }
}

// Stacks of at least this many problems are rebuilt from their running
// problems once half of them have stopped.
constexpr int kRestackMin = 8;

// Per-problem state of a lockstep solve that outlives one stack (restacking).
struct LockState {
  std::vector<int> active, k;
  std::vector<double> J, g02, amem;
  std::vector<reg_solve_report> R;
  explicit LockState(int n) : active(n, 1), k(n, 0), J(n, 0.0), g02(n, 0.0), amem(n, 1.0), R(n) {
    for (auto& r : R) std::memset(&r, 0, sizeof(r));
  }
};

// Runs the lockstep outer loop on the stack in c; slot q of the stack is
// problem S[slot[q]]. Returns true when it stops early so that the caller can
// restack the remaining problems: at the start of an outer iteration, when at
// most half of a stack of at least `restack_min` problems is still running.
// ---------------------------------------------------------------------------
// Device-driven loops of the lockstep solve. The PCG iteration and the Armijo
// trial of all problems of a stack run as CUDA graphs with conditional nodes:
// a WHILE node whose body runs a one-block check kernel (which stops the
// problems that are done and sets the loop conditions on the device) and an
// IF node holding one iteration (matvec, per-problem reductions into device
// rows, step lengths, vector updates). The host launches one graph per loop
// and reads the per-problem scalars back once per outer iteration. Every loop
// is bounded: PCG by kLockCap iterations per launch (the host relaunches while
// problems run and the iteration cap allows), the line search by the number
// of trials.
// ---------------------------------------------------------------------------
constexpr int kLockCap = 256;

// objective parts of stacked problems, unscaled, into device rows
void objective_seg_dev(reg_ctx* c, const double* v, double* d2_dev, double* r2_dev) {
  const long N = c->N();
  const int B = c->g.B;
  Work<double>& w = c->w64;
  REG_CUDA(cudaMemcpyAsync(w.m.get(N), c->mT.p, N * sizeof(double), cudaMemcpyDeviceToDevice, c->s));
  state_steps<double>(c, v, 0, c->n_t, nullptr, nullptr, 0, nullptr);
  double* scr = c->seg_scr.get(seg_scratch_doubles(B));
  seg_sqdiff_dev(c->mR.p, w.m.p, 1, B, c->g.N1, scr, c->s, d2_dev);
  double* Rv = c->tmpB.get(c->ncdN());
  tail(c, v, nullptr, Rv);
  seg_dot_dev(v, Rv, c->n_c * c->d, B, c->g.N1, scr, c->s, r2_dev);
}

// A WHILE loop in graph G around [check kernel -> IF(one iteration)].
void add_bounded_loop(cudaGraph_t G, cudaStream_t s,
                      const std::function<void(cudaGraphConditionalHandle, cudaGraphConditionalHandle)>& check,
                      const std::function<void()>& body) {
  cudaGraphConditionalHandle hw, hi;
  REG_CUDA(cudaGraphConditionalHandleCreate(&hw, G, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams wp{};
  wp.type = cudaGraphNodeTypeConditional;
  wp.conditional.handle = hw;
  wp.conditional.type = cudaGraphCondTypeWhile;
  wp.conditional.size = 1;
  cudaGraphNode_t wn;
  REG_CUDA(cudaGraphAddNode(&wn, G, nullptr, nullptr, 0, &wp));
  cudaGraph_t wbody = wp.conditional.phGraph_out[0];
  REG_CUDA(cudaGraphConditionalHandleCreate(&hi, wbody, 0, cudaGraphCondAssignDefault));
  cudaGraph_t done = nullptr;
  REG_CUDA(cudaStreamBeginCaptureToGraph(s, wbody, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  try {
    check(hi, hw);
    cudaStreamCaptureStatus st;
    cudaGraph_t cg = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    REG_CUDA(cudaStreamGetCaptureInfo(s, &st, nullptr, &cg, &deps, nullptr, &nd));
    cudaGraphNodeParams ip{};
    ip.type = cudaGraphNodeTypeConditional;
    ip.conditional.handle = hi;
    ip.conditional.type = cudaGraphCondTypeIf;
    ip.conditional.size = 1;
    cudaGraphNode_t in;
    REG_CUDA(cudaGraphAddNode(&in, cg, deps, nullptr, nd, &ip));
    REG_CUDA(cudaStreamUpdateCaptureDependencies(s, &in, nullptr, 1, cudaStreamSetCaptureDependencies));
    REG_CUDA(cudaStreamEndCapture(s, &done));
    REG_CUDA(cudaStreamBeginCaptureToGraph(s, ip.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                           cudaStreamCaptureModeThreadLocal));
    body();
    REG_CUDA(cudaStreamEndCapture(s, &done));
  } catch (...) {
    cudaStreamCaptureStatus st;
    if (cudaStreamIsCapturing(s, &st) == cudaSuccess && st != cudaStreamCaptureStatusNone)
      cudaStreamEndCapture(s, &done);
    (void)cudaGetLastError();
    throw;
  }
}

size_t lock_signature(reg_ctx* c, const double* v) {
  size_t h = graph_signature(c);
  const void* ptrs[] = {v, c->sv_g.p, c->sv_s.p, c->sv_r.p, c->sv_z.p, c->sv_p.p, c->sv_Hp.p, c->sv_vt.p,
                        c->lk.p, c->lkc.p, c->seg_scr.p, c->tmpB.p, c->mT.p, c->mR.p};
  for (const void* p : ptrs) h = (h ^ (size_t)p) * 1099511628211ull;
  return h;
}

// Builds (once per stack and buffer set) the PCG and line-search graphs.
// Returns false when the runtime refuses them (the host-driven loops run).
bool build_lock_graphs(reg_ctx* c, double* v, const reg_solve_opts& o, long maxit) {
  const size_t sig = lock_signature(c, v);
  if (c->lk_state == 1 && sig == c->lk_sig) return true;
  if (c->lk_state == -1) return false;
  if (c->lk_pcg) cudaGraphExecDestroy(c->lk_pcg);
  if (c->lk_ls) cudaGraphExecDestroy(c->lk_ls);
  c->lk_pcg = c->lk_ls = nullptr;
  const int B = c->g.B, K = c->n_c * c->d;
  const long N1 = c->g.N1, n = c->ncdN();
  double* g = c->sv_g.p;
  double* sv = c->sv_s.p;
  double* r = c->sv_r.p;
  double* z = c->sv_z.p;
  double* p = c->sv_p.p;
  double* Hp = c->sv_Hp.p;
  double* vt = c->sv_vt.p;
  double* lk = c->lk.p;
  int* ctl = c->lkc.p;
  double* scr = c->seg_scr.get(seg_scratch_doubles(B));
  auto row = [&](int slot) { return lk + (long)slot * B; };
  const int cap_it = (int)std::min<long>(maxit, 1L << 30);
  (void)n;
  cudaGraph_t G1 = nullptr, G2 = nullptr;
  try {
    REG_CUDA(cudaGraphCreate(&G1, 0));
    add_bounded_loop(
        G1, c->s,
        [&](cudaGraphConditionalHandle hi, cudaGraphConditionalHandle hw) {
          lk_pcg_check(lk, ctl, B, kLockCap, cap_it, (unsigned long long)hi, (unsigned long long)hw, c->s);
        },
        [&]() {
          hessvec_body(c, p, Hp);
          seg_dot_dev(p, Hp, K, B, N1, scr, c->s, row(LK_PHP));
          lk_pcg_alpha(lk, ctl, B, c->s);
          lincomb_seg(row(LK_NEGC), p, row(LK_KEEP), sv, sv, K, B, N1, c->s);
          lincomb_seg(row(LK_A), p, row(LK_ONE), sv, sv, K, B, N1, c->s);
          lincomb_seg(row(LK_A), Hp, row(LK_ONE), r, r, K, B, N1, c->s);
          precond(c, r, z);
          seg_dot_dev(r, z, K, B, N1, scr, c->s, row(LK_RZN));
          lk_pcg_beta(lk, ctl, B, c->s);
          lincomb_seg(row(LK_MZ), z, row(LK_BT), p, p, K, B, N1, c->s);
          seg_dot_dev(r, r, K, B, N1, scr, c->s, row(LK_RN2));
        });
    REG_CUDA(cudaGraphInstantiate(&c->lk_pcg, G1, 0));
    REG_CUDA(cudaGraphCreate(&G2, 0));
    add_bounded_loop(
        G2, c->s,
        [&](cudaGraphConditionalHandle hi, cudaGraphConditionalHandle hw) {
          lk_ls_check(lk, ctl, B, o.max_backtracks, (unsigned long long)hi, (unsigned long long)hw, c->s);
        },
        [&]() {
          lincomb_seg(row(LK_ONE), v, row(LK_ALPHA), sv, vt, K, B, N1, c->s);
          objective_seg_dev(c, vt, row(LK_D2), row(LK_R2));
          lk_ls_armijo(lk, B, c->hd, o.armijo_c1, o.backtrack, c->s);
        });
    REG_CUDA(cudaGraphInstantiate(&c->lk_ls, G2, 0));
  } catch (const CudaError& e) {
    if (G1) cudaGraphDestroy(G1);
    if (G2) cudaGraphDestroy(G2);
    if (c->lk_pcg) cudaGraphExecDestroy(c->lk_pcg);
    if (c->lk_ls) cudaGraphExecDestroy(c->lk_ls);
    c->lk_pcg = c->lk_ls = nullptr;
    (void)cudaGetLastError();
    c->lk_state = -1;
    return false;
  }
  cudaGraphDestroy(G1);
  cudaGraphDestroy(G2);
  c->lk_sig = sig;
  c->lk_state = 1;
  return true;
}

bool solve_lockstep(reg_ctx* c, double* v, const reg_solve_opts& o, LockState& S, const std::vector<int>& slot,
                    bool resume, int restack_min) {
  const int B = c->g.B;
  const long n = c->ncdN();
  double* g = c->sv_g.get(n);
  double* s = c->sv_s.get(n);
  double* r = c->sv_r.get(n);
  double* z = c->sv_z.get(n);
  double* p = c->sv_p.get(n);
  double* Hp = c->sv_Hp.get(n);
  double* vt = c->sv_vt.get(n);
  Seg sg(c, c->n_c * c->d);
  const long maxit = o.pcg_maxit > 0 ? o.pcg_maxit : n / B;
  std::vector<double> dist, regt, J(B), ginf, g2, g02(B), zero(B, 0.0), one(B, 1.0), tmp, tmp2;
  std::vector<int> active(B), k(B);
  std::vector<double> amem(B);
  std::vector<reg_solve_report*> Rp(B);
  for (int q = 0; q < B; ++q) {
    active[q] = S.active[slot[q]];
    k[q] = S.k[slot[q]];
    amem[q] = S.amem[slot[q]];
    g02[q] = S.g02[slot[q]];
    Rp[q] = &S.R[slot[q]];
  }
  struct Sync {  // the per-problem state back into S on every exit
    LockState& S;
    const std::vector<int>& slot;
    std::vector<int>& active;
    std::vector<int>& k;
    std::vector<double>& J;
    std::vector<double>& amem;
    ~Sync() {
      for (size_t q = 0; q < slot.size(); ++q) {
        S.active[slot[q]] = active[q];
        S.k[slot[q]] = k[q];
        S.J[slot[q]] = J[q];
        S.amem[slot[q]] = amem[q];
      }
    }
  } sync{S, slot, active, k, J, amem};
  auto R = [&](int q) -> reg_solve_report& { return *Rp[q]; };
  auto finite_or_fail = [&](int q, double x) {
    if (active[q] && !std::isfinite(x)) {
      active[q] = 0;
      R(q).status = REG_ENONFINITE;
    }
  };
  // final measures of the problems that have stopped (all, at the end)
  auto finalize = [&](bool all) {
    std::vector<double> base(B), cf;
    Seg one1(c, 1);
    seg_sqdiff(c->mT.p, c->mR.p, 1, B, c->g.N1, one1.scr, c->s, base.data());
    cfl_seg(c, v, cf);
    for (int q = 0; q < B; ++q) {
      if (!all && active[q]) continue;
      R(q).outer = k[q];
      R(q).J = J[q];
      R(q).dist_rel = base[q] > 0 ? (2.0 * dist[q] / c->hd) / base[q] : 0.0;
      R(q).cfl = cf[q];
    }
  };
  gradient_seg(c, v, g, dist, regt);
  // the device-driven loops (Krylov method without CFL halving); one ordinary
  // matvec first allocates every buffer and settles the autotuned passes
  bool graph_mode = false;
  {
    const char* env = getenv("REG_LOCKSTEP_GRAPHS");
    if (o.method == REG_METHOD_KRYLOV && !(o.cfl_max > 0) && !(env && env[0] == '0')) {
      c->lk.get((size_t)LK_COUNT * B);
      c->lkc.get(LC_COUNT);
      if (c->lk_state == 0) hessvec_body(c, g, Hp);
      graph_mode = build_lock_graphs(c, v, o, maxit);
    }
    for (int q = 0; q < B; ++q)
      if (graph_mode) R(q).device_loops = 1;
  }
  if (!resume) {
    sg.maxabs(g, ginf);
    sg.dot(g, g, tmp);
    sg.maxabs(v, tmp2);
    for (int q = 0; q < B; ++q) {
      J[q] = dist[q] + regt[q];
      R(q).n_pde = 2;
      R(q).J0 = J[q];
      R(q).g0_inf = ginf[q];
      R(q).v_inf = tmp2[q];
      R(q).alpha_mem = 1.0;
      g02[q] = std::sqrt(tmp[q]);
      S.g02[slot[q]] = g02[q];
      finite_or_fail(q, J[q] + tmp[q]);
    }
  } else {
    for (int q = 0; q < B; ++q) J[q] = dist[q] + regt[q];
  }
  for (;;) {
    sg.maxabs(g, ginf);
    sg.dot(g, g, tmp);
    g2.assign(B, 0.0);
    int live = 0;
    for (int q = 0; q < B; ++q) {
      g2[q] = std::sqrt(tmp[q]);
      if (!active[q]) continue;
      R(q).g_inf = ginf[q];
      R(q).J = J[q];
      bool maxed = false;
      if (stop_test(o, R(q), k[q], ginf[q], maxed)) {
        active[q] = 0;
        R(q).status = maxed ? REG_EMAXIT : REG_OK;
      } else {
        ++live;
      }
    }
    if (!live) break;
    if (B >= restack_min && 2 * live <= B) {  // restack the running problems
      finalize(false);
      return true;
    }
    std::vector<double> act(B);
    for (int q = 0; q < B; ++q) act[q] = active[q] ? 1.0 : 0.0;
    std::vector<double> slope, alpha(B, 0.0), Jt(B, 0.0);
    if (graph_mode) {
      // PCG and line search of every problem on the device (see build_lock_graphs)
      const int K = c->n_c * c->d;
      const long N1 = c->g.N1;
      double* lk = c->lk.p;
      int* ctl = c->lkc.p;
      double* scr = c->seg_scr.get(seg_scratch_doubles(B));
      auto row = [&](int slot) { return lk + (long)slot * B; };
      std::vector<double>& h = c->lkh;
      h.assign((size_t)LK_COUNT * B, 0.0);
      for (int q = 0; q < B; ++q) {
        h[(size_t)LK_ACT * B + q] = active[q] ? 1.0 : 0.0;
        h[(size_t)LK_G2 * B + q] = g2[q];
        h[(size_t)LK_G02 * B + q] = g02[q];
        h[(size_t)LK_J * B + q] = J[q];
      }
      REG_CUDA(cudaMemcpyAsync(lk, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice, c->s));
      lk_pcg_init(lk, ctl, B, c->s);
      REG_CUDA(cudaMemsetAsync(s, 0, n * sizeof(double), c->s));
      REG_CUDA(cudaMemcpyAsync(r, g, n * sizeof(double), cudaMemcpyDeviceToDevice, c->s));
      precond(c, r, z);
      lincomb_seg(row(LK_MONE), z, row(LK_ZERO), z, p, K, B, N1, c->s);
      seg_dot_dev(r, z, K, B, N1, scr, c->s, row(LK_RZ));
      seg_dot_dev(r, r, K, B, N1, scr, c->s, row(LK_RN2));
      for (;;) {  // each launch runs at most kLockCap iterations
        REG_CUDA(cudaMemsetAsync(ctl + LC_IT, 0, sizeof(int), c->s));
        REG_CUDA(cudaGraphLaunch(c->lk_pcg, c->s));
        int hc[LC_COUNT];
        REG_CUDA(cudaMemcpyAsync(hc, ctl, sizeof(hc), cudaMemcpyDeviceToHost, c->s));
        REG_CUDA(cudaStreamSynchronize(c->s));
        if (!(hc[LC_ON] && hc[LC_PIT] < maxit && hc[LC_IT] >= kLockCap)) break;
      }
      seg_dot_dev(g, s, K, B, N1, scr, c->s, row(LK_SLOPE));
      lk_ls_init(lk, ctl, B, c->hd, c->s);
      REG_CUDA(cudaGraphLaunch(c->lk_ls, c->s));
      lk_ls_final(lk, B, REG_ELINESEARCH, c->s);
      REG_CUDA(cudaMemcpyAsync(h.data(), lk, h.size() * sizeof(double), cudaMemcpyDeviceToHost, c->s));
      REG_CUDA(cudaStreamSynchronize(c->s));
      for (int q = 0; q < B; ++q) {
        active[q] = h[(size_t)LK_ACT * B + q] != 0.0;
        const int st = (int)h[(size_t)LK_STATUS * B + q];
        if (st) R(q).status = st;
        R(q).pcg_iters += (long)h[(size_t)LK_PCG * B + q];
        R(q).matvecs += (long)h[(size_t)LK_MV * B + q];
        R(q).n_pde += (long)h[(size_t)LK_NPDE * B + q];
        R(q).ls_trials += (int)h[(size_t)LK_LS * B + q];
        alpha[q] = h[(size_t)LK_ALPHA * B + q];
      }
    } else if (o.method == REG_METHOD_PICARD) {
      precond(c, g, s);
      std::vector<double> sc(B);
      for (int q = 0; q < B; ++q) sc[q] = active[q] ? (o.step_memory ? -amem[q] : -1.0) : 0.0;
      sg.comb(zero, s, sc, s, s);
    } else {
      // PCG on H s = -g from s = 0, all active problems at once
      std::vector<double> eta(B), rz, rzn, pHp, rn2, on(B);
      for (int q = 0; q < B; ++q) {
        eta[q] = std::min(0.5, std::sqrt(g2[q] / g02[q]));
        on[q] = active[q];
      }
      REG_CUDA(cudaMemsetAsync(s, 0, n * sizeof(double), c->s));
      REG_CUDA(cudaMemcpyAsync(r, g, n * sizeof(double), cudaMemcpyDeviceToDevice, c->s));
      precond(c, r, z);
      sg.comb(std::vector<double>(B, -1.0), z, zero, z, p);
      sg.dot(r, z, rz);
      for (long it = 0; it < maxit; ++it) {
        sg.dot(r, r, rn2);
        int running = 0;
        for (int q = 0; q < B; ++q) {
          if (!on[q]) continue;
          finite_or_fail(q, rn2[q]);
          if (!active[q] || std::sqrt(rn2[q]) <= eta[q] * g2[q]) on[q] = 0;
          else ++running;
        }
        if (!running) break;
        hessvec(c, p, Hp);
        sg.dot(p, Hp, pHp);
        std::vector<double> a(B, 0.0), cs(B, 1.0), copy_p(B, 0.0);
        bool any_copy = false;
        for (int q = 0; q < B; ++q) {
          if (!on[q]) continue;
          R(q).matvecs += 1;
          R(q).n_pde += 2;
          R(q).pcg_iters += 1;
          finite_or_fail(q, pHp[q]);
          if (!active[q]) {
            on[q] = 0;
          } else if (pHp[q] <= 0.0) {
            if (it == 0) {
              copy_p[q] = 1.0;
              any_copy = true;
            }
            on[q] = 0;
          } else {
            a[q] = rz[q] / pHp[q];
          }
        }
        if (any_copy) {  // negative curvature at the first step: the steepest-descent direction
          std::vector<double> keep(B);
          for (int q = 0; q < B; ++q) keep[q] = copy_p[q] != 0.0 ? 0.0 : 1.0;
          sg.comb(copy_p, p, keep, s, s);
        }
        sg.comb(a, p, one, s, s);
        sg.comb(a, Hp, one, r, r);
        precond(c, r, z);
        sg.dot(r, z, rzn);
        std::vector<double> mz(B, 0.0), bt(B, 1.0);
        for (int q = 0; q < B; ++q)
          if (on[q]) {
            mz[q] = -1.0;
            bt[q] = rzn[q] / rz[q];
            rz[q] = rzn[q];
          }
        sg.comb(mz, z, bt, p, p);
      }
    }
    // keep each step inside the CFL bound by halving it (Sec. 3.3.5)
    if (!graph_mode && o.cfl_max > 0) {
      std::vector<int> halvings(B, 0);
      for (;;) {
        sg.comb(one, v, one, s, vt);
        std::vector<double> cf;
        cfl_seg(c, vt, cf);
        std::vector<double> h(B, 1.0);
        bool any = false;
        for (int q = 0; q < B; ++q) {
          if (!active[q] || cf[q] <= o.cfl_max) continue;
          if (++halvings[q] > 30) {
            active[q] = 0;
            R(q).status = REG_ECFL;
            h[q] = 0.0;  // no step
          } else {
            h[q] = 0.5;
            R(q).cfl_halvings += 1;
          }
          any = true;
        }
        if (!any) break;
        sg.comb(zero, s, h, s, s);
      }
    }
    // Armijo backtracking from alpha = 1, per problem
    if (!graph_mode) {
    sg.dot(g, s, slope);
    for (double& x : slope) x *= c->hd;
    std::vector<int> searching(B, 0);
    int nsearch = 0;
    for (int q = 0; q < B; ++q)
      if (active[q]) {
        alpha[q] = 1.0;
        searching[q] = 1;
        ++nsearch;
      }
    for (int t = 0; t < o.max_backtracks && nsearch; ++t) {
      sg.comb(one, v, alpha, s, vt);
      std::vector<double> d2, r2;
      objective_seg(c, vt, d2, r2);
      for (int q = 0; q < B; ++q) {
        if (!searching[q]) continue;
        R(q).ls_trials += 1;
        R(q).n_pde += 1;
        Jt[q] = d2[q] + r2[q];
        if (std::isfinite(Jt[q]) && Jt[q] <= J[q] + o.armijo_c1 * alpha[q] * slope[q]) {
          searching[q] = 0;
          --nsearch;
        } else {
          alpha[q] *= o.backtrack;
        }
      }
    }
    for (int q = 0; q < B; ++q)
      if (searching[q]) {  // no sufficient decrease: the problem keeps its iterate
        active[q] = 0;
        R(q).status = REG_ELINESEARCH;
        alpha[q] = 0.0;
      }
    }
    for (int q = 0; q < B; ++q) {
      if (!active[q]) alpha[q] = 0.0;
      if (active[q] && o.method == REG_METHOD_PICARD && o.step_memory)
        amem[q] = (alpha[q] == 1.0) ? 2.0 * amem[q] : amem[q] * alpha[q];
      R(q).alpha_mem = amem[q];
    }
    sg.comb(one, v, alpha, s, vt);
    sg.comb(one, vt, std::vector<double>(B, -1.0), v, r);  // v_k - v_{k-1}
    std::vector<double> dv, vin;
    sg.maxabs(r, dv);
    REG_CUDA(cudaMemcpyAsync(v, vt, n * sizeof(double), cudaMemcpyDeviceToDevice, c->s));
    sg.maxabs(v, vin);
    std::vector<int> stepped = active;
    for (int q = 0; q < B; ++q)
      if (stepped[q]) {
        R(q).dv_inf = dv[q];
        R(q).v_inf = vin[q];
        R(q).J_prev = J[q];
      }
    gradient_seg(c, v, g, dist, regt);
    for (int q = 0; q < B; ++q) {
      if (!stepped[q]) continue;
      J[q] = dist[q] + regt[q];
      R(q).n_pde += 2;
      k[q] += 1;
      finite_or_fail(q, J[q]);
    }
  }
  finalize(true);
  return false;
}

}  // namespace

void reg::set_thread_error(const std::string& msg) { g_create_error = msg; }

namespace {

// a tile copy of the TMA column pass that never landed leaves garbage: fail the call
void check_copies(reg_ctx* c) {
  if (take_tma_timeouts_f32(c->s) + take_tma_timeouts_f64(c->s) > 0)
    throw StatusError{REG_ETIMEOUT, "a tile copy of the column pass timed out"};
}

reg_status fail(reg_ctx* c, int st, const std::string& msg) {
  if (c) c->err = msg;
  else g_create_error = msg;
  return (reg_status)st;
}

}  // namespace

#define API_BEGIN(ctx)                                          \
  if (!(ctx)) return fail(nullptr, REG_EINVAL, "null context"); \
  reg_ctx* c_ = (ctx);                                          \
  c_->err.clear();                                              \
  tl_prof = c_->prof.mask ? &c_->prof : nullptr;                \
  try {
#define API_END                                                                                       \
  check_copies(c_);                                                                                   \
  }                                                                                                   \
  catch (const StatusError& e) {                                                                      \
    return fail(c_, e.status, e.what);                                                                \
  }                                                                                                   \
  catch (const CudaError& e) {                                                                        \
    return fail(c_, e.code == cudaErrorMemoryAllocation ? REG_ENOMEM : REG_ECUDA, e.what);            \
  }                                                                                                   \
  catch (const std::bad_alloc&) {                                                                     \
    return fail(c_, REG_ENOMEM, "host allocation failed");                                            \
  }                                                                                                   \
  return REG_OK;

namespace {

// A context on B stacked problems of one shape (B = 1: the ordinary context).
// Arguments are validated by the caller. Throws on failure.
reg_ctx* create_ctx(int d, const int64_t* n, int n_t, int n_c, double beta, int reg_type, int stokes, int precision,
                    int ckpt_every, void* cuda_stream, int batch) {
  Grid g = make_grid(d, n, batch);
  std::unique_ptr<reg_ctx> holder(new reg_ctx());
  reg_ctx* c = holder.get();
  c->d = d;
  c->g = g;
  c->n_t = n_t;
  c->n_c = n_c;
  c->beta = beta;
  c->rtype = reg_type;
  c->stokes = stokes;
  c->prec = precision;
  c->ckpt = ckpt_every;
  c->s = (cudaStream_t)cuda_stream;
  c->graphs = c->s != nullptr;  // a context with its own stream replays its matvec as a CUDA graph
  for (int i = 0; i < d; ++i) c->hd *= 2.0 * M_PI / g.n[i];
  c->bnode.resize((size_t)(n_t + 1) * n_c);
  for (int j = 0; j <= n_t; ++j) cheb_values(n_c, (double)j / n_t, &c->bnode[(size_t)j * n_c]);
  c->Cg.resize(n_c * n_c);
  for (int a = 0; a < n_c; ++a)
    for (int b = 0; b < n_c; ++b) c->Cg[a * n_c + b] = cheb_gram_entry(a, b);
  if (!invert_small(n_c, c->Cg, c->Ci)) throw StatusError{REG_EINVAL, "singular Gram matrix"};
  REG_CUDA(cudaMemcpy(c->Cg_dev.get(n_c * n_c), c->Cg.data(), n_c * n_c * sizeof(double), cudaMemcpyHostToDevice));
  REG_CUDA(cudaMemcpy(c->Ci_dev.get(n_c * n_c), c->Ci.data(), n_c * n_c * sizeof(double), cudaMemcpyHostToDevice));
  c->sp64.reset(new Spectral<double>(g, c->s));
  if (precision == REG_MIXED) c->sp32.reset(new Spectral<float>(g, c->s));
  return holder.release();
}

}  // namespace

extern "C" {

reg_status reg_create(reg_ctx** out, int d, const int64_t* n, int n_t, int n_c, double beta, int reg_type, int stokes,
                      int precision, int ckpt_every, void* cuda_stream) {
  if (!out) return fail(nullptr, REG_EINVAL, "out is null");
  *out = nullptr;
  if (!n) return fail(nullptr, REG_EINVAL, "n is null");
  if (n_t < 1) return fail(nullptr, REG_EINVAL, "n_t must be >= 1");
  if (n_c < 1 || n_c > 16) return fail(nullptr, REG_EINVAL, "n_c must be in [1, 16]");
  if (!(beta > 0.0) || !std::isfinite(beta)) return fail(nullptr, REG_EINVAL, "beta must be positive and finite");
  if (reg_type != REG_H1 && reg_type != REG_H2) return fail(nullptr, REG_EINVAL, "reg_type must be REG_H1 or REG_H2");
  if (stokes != 0 && stokes != 1) return fail(nullptr, REG_EINVAL, "stokes must be 0 or 1");
  if (precision != REG_FP64 && precision != REG_MIXED) return fail(nullptr, REG_EINVAL, "bad precision");
  if (ckpt_every < 0 || (ckpt_every > 0 && n_t % ckpt_every != 0))
    return fail(nullptr, REG_EINVAL, "ckpt_every must be 0 or divide n_t");
  try {
    *out = create_ctx(d, n, n_t, n_c, beta, reg_type, stokes, precision, ckpt_every, cuda_stream, 1);
  } catch (const StatusError& e) {
    return fail(nullptr, e.status, e.what);
  } catch (const CudaError& e) {
    return fail(nullptr, e.code == cudaErrorMemoryAllocation ? REG_ENOMEM : REG_ECUDA, e.what);
  } catch (const std::bad_alloc&) {
    return fail(nullptr, REG_ENOMEM, "host allocation failed");
  }
  return REG_OK;
}

reg_status reg_destroy(reg_ctx* ctx) {
  if (!ctx) return REG_OK;
  cudaStreamSynchronize(ctx->s);
  delete ctx;
  return REG_OK;
}

const char* reg_last_error(const reg_ctx* ctx) { return ctx ? ctx->err.c_str() : g_create_error.c_str(); }

reg_status reg_set_quadrature(reg_ctx* ctx, int quadrature) {
  API_BEGIN(ctx)
  if (quadrature != REG_QUAD_TRAPEZOID && quadrature != REG_QUAD_DISCRETE)
    throw StatusError{REG_EINVAL, "bad quadrature"};
  if (quadrature == REG_QUAD_DISCRETE && c_->hess == REG_HESS_NEWTON)
    throw StatusError{REG_EINVAL, "the full Newton Hessian uses the trapezoid quadrature"};
  c_->quad = quadrature;
  c_->ready = false;
  API_END
}

reg_status reg_set_hessian(reg_ctx* ctx, int kind) {
  API_BEGIN(ctx)
  if (kind != REG_HESS_GN && kind != REG_HESS_NEWTON) throw StatusError{REG_EINVAL, "bad Hessian kind"};
  if (kind == REG_HESS_NEWTON && c_->quad != REG_QUAD_TRAPEZOID)
    throw StatusError{REG_EINVAL, "the full Newton Hessian uses the trapezoid quadrature"};
  c_->hess = kind;
  c_->ready = false;
  API_END
}

reg_status reg_set_images(reg_ctx* ctx, const double* m_T, const double* m_R) {
  API_BEGIN(ctx)
  const long N = c_->N();
  const double* a = input_ptr(c_, m_T, N, 0);
  const double* b = input_ptr(c_, m_R, N, 1);
  REG_CUDA(cudaMemcpyAsync(c_->mT.get(N), a, N * sizeof(double), cudaMemcpyDeviceToDevice, c_->s));
  REG_CUDA(cudaMemcpyAsync(c_->mR.get(N), b, N * sizeof(double), cudaMemcpyDeviceToDevice, c_->s));
  REG_CUDA(cudaStreamSynchronize(c_->s));
  c_->have_images = true;
  c_->ready = false;
  API_END
}

reg_status reg_objective(reg_ctx* ctx, const double* v, double* J_out, double* parts) {
  API_BEGIN(ctx)
  if (!J_out) throw StatusError{REG_EINVAL, "J_out is null"};
  const double* vd = input_ptr(c_, v, c_->ncdN(), 0);
  double p[2];
  objective(c_, vd, p);
  check_finite(p[0] + p[1], "objective");
  *J_out = p[0] + p[1];
  if (parts) {
    parts[0] = p[0];
    parts[1] = p[1];
  }
  API_END
}

reg_status reg_gradient(reg_ctx* ctx, const double* v, double* g, double* J_out) {
  API_BEGIN(ctx)
  const double* vd = input_ptr(c_, v, c_->ncdN(), 0);
  Output o(c_, g, c_->ncdN(), c_->stage_out);
  double p[2];
  gradient(c_, vd, o.dev, p);
  o.finish();
  if (J_out) *J_out = p[0] + p[1];
  API_END
}

reg_status reg_linearize(reg_ctx* ctx, const double* v) {
  API_BEGIN(ctx)
  const double* vd = input_ptr(c_, v, c_->ncdN(), 0);
  set_point(c_, vd);
  prepare_mixed(c_);
  REG_CUDA(cudaStreamSynchronize(c_->s));
  c_->ready = true;
  API_END
}

reg_status reg_hessvec(reg_ctx* ctx, const double* vt, double* Hvt) {
  API_BEGIN(ctx)
  const double* vd = input_ptr(c_, vt, c_->ncdN(), 0);
  Output o(c_, Hvt, c_->ncdN(), c_->stage_out);
  hessvec(c_, vd, o.dev);
  o.finish();
  API_END
}

reg_status reg_precond(reg_ctx* ctx, const double* r, double* z) {
  API_BEGIN(ctx)
  const double* rd = input_ptr(c_, r, c_->ncdN(), 0);
  Output o(c_, z, c_->ncdN(), c_->stage_out);
  precond(c_, rd, o.dev);
  o.finish();
  API_END
}

reg_status reg_regularization(reg_ctx* ctx, const double* v, double* out) {
  API_BEGIN(ctx)
  const double* vd = input_ptr(c_, v, c_->ncdN(), 0);
  Output o(c_, out, c_->ncdN(), c_->stage_out);
  tail(c_, vd, nullptr, o.dev);
  o.finish();
  API_END
}

reg_status reg_transport(reg_ctx* ctx, const double* v, const double* m0, double* m1) {
  API_BEGIN(ctx)
  const long N = c_->N();
  const double* vd = input_ptr(c_, v, c_->ncdN(), 0);
  const double* md = input_ptr(c_, m0, N, 1);
  Output o(c_, m1, N, c_->stage_out);
  Work<double>& w = c_->w64;
  REG_CUDA(cudaMemcpyAsync(w.m.get(N), md, N * sizeof(double), cudaMemcpyDeviceToDevice, c_->s));
  state_steps<double>(c_, vd, 0, c_->n_t, nullptr, nullptr, 0, nullptr);
  REG_CUDA(cudaMemcpyAsync(o.dev, w.m.p, N * sizeof(double), cudaMemcpyDeviceToDevice, c_->s));
  o.finish();
  API_END
}

reg_status reg_transport_adjoint(reg_ctx* ctx, const double* v, const double* m0, const double* G, double* grad_v,
                                 double* grad_m0) {
  API_BEGIN(ctx)
  const long N = c_->N();
  const double* vd = input_ptr(c_, v, c_->ncdN(), 0);
  const double* md = input_ptr(c_, m0, N, 1);
  const double* Gd = input_ptr(c_, G, N, 2);
  c_->ready = false;  // the stored state now belongs to (v, m0)
  double* vc = c_->tmpA.get(c_->ncdN());
  REG_CUDA(cudaMemcpyAsync(vc, vd, c_->ncdN() * sizeof(double), cudaMemcpyDeviceToDevice, c_->s));
  state_solve_store<double>(c_, vc, md);
  Work<double>& w = c_->w64;
  lincomb_t<double>(-1.0, Gd, 0.0, nullptr, w.lam.get(N), N, c_->s);  // lam_1 = -G
  double* f = c_->f.get(c_->ncdN());
  adjoint_solve<double>(c_, vc, f);
  if (grad_v) {
    Output o(c_, grad_v, c_->ncdN(), c_->stage_out);
    REG_CUDA(cudaMemcpyAsync(o.dev, f, c_->ncdN() * sizeof(double), cudaMemcpyDeviceToDevice, c_->s));
    o.finish();
  }
  if (grad_m0) {
    Output o(c_, grad_m0, N, c_->stage_out);
    lincomb_t<double>(-1.0, w.lam.p, 0.0, nullptr, o.dev, N, c_->s);
    o.finish();
  }
  REG_CUDA(cudaStreamSynchronize(c_->s));
  API_END
}

reg_status reg_detF(reg_ctx* ctx, const double* v, int substeps, double* stats_out, double* detF_out) {
  API_BEGIN(ctx)
  if (substeps < 1) throw StatusError{REG_EINVAL, "substeps must be >= 1"};
  if (!stats_out) throw StatusError{REG_EINVAL, "stats is null"};
  const double* vd = input_ptr(c_, v, c_->ncdN(), 0);
  double st[4];
  if (detF_out) {
    Output o(c_, detF_out, c_->N(), c_->stage_out);
    detF(c_, vd, substeps, st, o.dev);
    o.finish();
  } else {
    detF(c_, vd, substeps, st, nullptr);
  }
  for (int i = 0; i < 4; ++i) stats_out[i] = st[i];
  API_END
}

reg_status reg_detF_refined(reg_ctx* ctx, const double* v, int substeps, int refine, double* stats_out,
                            double* detF_out) {
  API_BEGIN(ctx)
  if (substeps < 1) throw StatusError{REG_EINVAL, "substeps must be >= 1"};
  if (refine != 1 && refine != 2 && refine != 4) throw StatusError{REG_EINVAL, "refine must be 1, 2 or 4"};
  if (!stats_out) throw StatusError{REG_EINVAL, "stats is null"};
  const double* vd = input_ptr(c_, v, c_->ncdN(), 0);
  long nfine = c_->N();
  for (int a = 0; a < c_->d; ++a) nfine *= refine;
  double st[4];
  if (detF_out) {
    Output o(c_, detF_out, nfine, c_->stage_out);
    detF_refined(c_, vd, substeps, refine, st, o.dev);
    o.finish();
  } else {
    detF_refined(c_, vd, substeps, refine, st, nullptr);
  }
  for (int i = 0; i < 4; ++i) stats_out[i] = st[i];
  API_END
}

reg_status reg_cfl(reg_ctx* ctx, const double* v, double* cfl_out) {
  API_BEGIN(ctx)
  if (!cfl_out) throw StatusError{REG_EINVAL, "cfl_out is null"};
  const double* vd = input_ptr(c_, v, c_->ncdN(), 0);
  *cfl_out = cfl(c_, vd);
  API_END
}

reg_status reg_grid_angle(reg_ctx* ctx, const double* v, int substeps, double* stats_out, double* angle_out) {
  API_BEGIN(ctx)
  if (substeps < 1) throw StatusError{REG_EINVAL, "substeps must be >= 1"};
  if (!stats_out) throw StatusError{REG_EINVAL, "stats is null"};
  const double* vd = input_ptr(c_, v, c_->ncdN(), 0);
  double dst[4], ast[4];
  if (angle_out) {
    Output o(c_, angle_out, c_->N(), c_->stage_out);
    deform_measures(c_, vd, substeps, dst, ast, nullptr, o.dev);
    o.finish();
  } else {
    deform_measures(c_, vd, substeps, dst, ast, nullptr, nullptr);
  }
  for (int i = 0; i < 4; ++i) stats_out[i] = ast[i];
  API_END
}

reg_status reg_displacement(reg_ctx* ctx, const double* v, double* u) {
  API_BEGIN(ctx)
  const double* vd = input_ptr(c_, v, c_->ncdN(), 0);
  Output o(c_, u, c_->dN(), c_->stage_out);
  if (o.dev == vd) throw StatusError{REG_EINVAL, "u may not alias v"};
  displacement(c_, vd, o.dev);
  o.finish();
  API_END
}

reg_status reg_smooth(reg_ctx* ctx, double sigma, const double* in, double* out) {
  API_BEGIN(ctx)
  if (!(sigma >= 0.0) || !std::isfinite(sigma)) throw StatusError{REG_EINVAL, "sigma must be finite and >= 0"};
  const double* id = input_ptr(c_, in, c_->N(), 0);
  Output o(c_, out, c_->N(), c_->stage_out);
  smooth(c_, sigma, id, o.dev);
  o.finish();
  API_END
}

reg_status reg_lanczos(reg_ctx* ctx, const double* q0, int k, int precond_flag, double* alpha, double* beta,
                       int* steps, double* ritz) {
  API_BEGIN(ctx)
  if (k < 1) throw StatusError{REG_EINVAL, "k must be >= 1"};
  if (!alpha || !beta || !steps) throw StatusError{REG_EINVAL, "null output argument"};
  if (!c_->ready) throw StatusError{REG_ENOTREADY, "no linearisation point: call reg_gradient or reg_linearize first"};
  const double* qd = input_ptr(c_, q0, c_->ncdN(), 0);
  int m = lanczos(c_, qd, k, precond_flag ? 1 : 0, alpha, beta);
  REG_CUDA(cudaStreamSynchronize(c_->s));
  *steps = m;
  if (ritz) tridiag_eigs(alpha, beta, m, ritz);
  API_END
}

reg_status reg_set_beta(reg_ctx* ctx, double beta) {
  API_BEGIN(ctx)
  if (!(beta > 0.0) || !std::isfinite(beta)) throw StatusError{REG_EINVAL, "beta must be positive and finite"};
  c_->beta = beta;
  API_END
}

reg_status reg_set_time_steps(reg_ctx* ctx, int n_t) {
  API_BEGIN(ctx)
  set_time_steps(c_, n_t);
  API_END
}

void reg_cont_opts_default(reg_cont_opts* o) {
  if (!o) return;
  o->beta0 = 1.0;
  o->beta_min = 1e-6;
  o->eps_F = 0.1;
  o->eps_theta = 0.0;
  o->beta_rtol = 0.05;
  o->dist_rtol = 1e-2;
  o->cfl_target = 0.0;
  o->detF_substeps = 1;
  o->max_solves = 50;
}

reg_status reg_continuation(reg_ctx* ctx, double* v_inout, const reg_solve_opts* solve_opts,
                            const reg_cont_opts* cont_opts, reg_cont_report* report) {
  API_BEGIN(ctx)
  if (!c_->have_images) throw StatusError{REG_EINVAL, "reg_set_images has not been called"};
  reg_solve_opts so;
  reg_solve_opts_default(&so);
  if (solve_opts) so = *solve_opts;
  reg_cont_opts co;
  reg_cont_opts_default(&co);
  if (cont_opts) co = *cont_opts;
  if (!v_inout) throw StatusError{REG_EINVAL, "v_inout is null"};
  Output io(c_, v_inout, c_->ncdN(), c_->stage_out);
  if (io.host)
    REG_CUDA(cudaMemcpyAsync(io.dev, v_inout, c_->ncdN() * sizeof(double), cudaMemcpyHostToDevice, c_->s));
  reg_cont_report R;
  continuation(c_, io.dev, so, co, R);
  io.finish();
  if (report) *report = R;
  API_END
}

reg_status reg_profile_begin(reg_ctx* ctx, unsigned kind_mask) {
  API_BEGIN(ctx)
  double ms[KK_COUNT], by[KK_COUNT];
  long cnt[KK_COUNT];
  c_->prof.collect(ms, by, cnt);  // drop anything left over
  c_->prof.mask = kind_mask;
  API_END
}

reg_status reg_profile_end(reg_ctx* ctx, double* ms, double* bytes, long* count) {
  API_BEGIN(ctx)
  double m[KK_COUNT], b[KK_COUNT];
  long n[KK_COUNT];
  c_->prof.collect(m, b, n);
  c_->prof.mask = 0;
  for (int k = 0; k < KK_COUNT; ++k) {
    if (ms) ms[k] = m[k];
    if (bytes) bytes[k] = b[k];
    if (count) count[k] = n[k];
  }
  API_END
}

reg_status reg_profile_flops(reg_ctx* ctx, double* flops) {
  API_BEGIN(ctx)
  if (!flops) throw StatusError{REG_EINVAL, "flops is null"};
  for (int k = 0; k < KK_COUNT; ++k) flops[k] = c_->prof.last_flops[k];
  API_END
}

long reg_launch_count(void) { return launch_count(); }

void reg_solve_opts_default(reg_solve_opts* o) {
  if (!o) return;
  o->grad_rtol = 1e-2;
  o->max_outer = 50;
  o->armijo_c1 = 1e-4;
  o->backtrack = 0.5;
  o->max_backtracks = 20;
  o->pcg_maxit = 0;
  o->cfl_max = 0.0;
  o->detF_substeps = 0;
  o->method = REG_METHOD_KRYLOV;
  o->step_memory = 1;
  o->stop_rule = REG_STOP_GRAD_REL;
  o->tau_J = 1e-3;
  o->detF_refine = 1;
}

reg_status reg_solve_lockstep(const reg_problem* problems, int count, int precision, const reg_solve_opts* opts,
                              reg_solve_report* reports, int max_stack) {
  if (!problems || count < 0 || max_stack < 0) {
    g_create_error = "reg_solve_lockstep: bad arguments";
    return REG_EINVAL;
  }
  if (count == 0) return REG_OK;
  if (precision != REG_FP64 && precision != REG_MIXED) {
    g_create_error = "reg_solve_lockstep: bad precision";
    return REG_EINVAL;
  }
  reg_solve_opts o;
  reg_solve_opts_default(&o);
  if (opts) o = *opts;
  // groups of one shape and time discretisation, in order of first appearance
  using GKey = std::tuple<int, int64_t, int64_t, int64_t, int, int, int, int>;
  std::map<GKey, std::vector<int>> groups;
  std::vector<GKey> order;
  for (int i = 0; i < count; ++i) {
    const reg_problem& p = problems[i];
    if ((p.d != 2 && p.d != 3) || p.n_t < 1 || p.n_c < 1 || p.n_c > 16 || !(p.beta > 0.0) ||
        (p.reg_type != REG_H1 && p.reg_type != REG_H2) || (p.stokes != 0 && p.stokes != 1) || !p.m_T || !p.m_R ||
        !p.v) {
      g_create_error = "reg_solve_lockstep: problem " + std::to_string(i) + " is invalid";
      return REG_EINVAL;
    }
    GKey k(p.d, p.n[0], p.n[1], p.d == 3 ? p.n[2] : 1, p.n_t, p.n_c, p.reg_type, p.stokes);
    if (!groups.count(k)) order.push_back(k);
    auto& list = groups[k];
    list.push_back(i);
  }
  // stacks of at most max_stack problems
  std::vector<std::vector<int>> stacks;
  for (const GKey& k : order) {
    const auto& list = groups[k];
    const int cap = max_stack > 0 ? max_stack : (int)list.size();
    for (size_t a = 0; a < list.size(); a += cap)
      stacks.emplace_back(list.begin() + a, list.begin() + std::min(list.size(), a + cap));
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    (void)cudaGetLastError();
    g_create_error = "reg_solve_lockstep: no CUDA device";
    return REG_ECUDA;
  }
  std::vector<int> status(stacks.size(), REG_OK);
  std::vector<std::string> errors(stacks.size());
  auto run = [&](size_t si) {
    cudaSetDevice(dev);
    const std::vector<int>& ids = stacks[si];
    const reg_problem& p0 = problems[ids[0]];
    cudaStream_t st = nullptr;
    reg_ctx* c = nullptr;
    auto t0 = std::chrono::steady_clock::now();
    try {
      REG_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
      LockState S((int)ids.size());
      std::vector<int> slot(ids.size());
      std::iota(slot.begin(), slot.end(), 0);
      bool resume = false;
      for (;;) {
        // a stack of the problems in `slot` (positions in ids), loaded from the callers' arrays
        const int B = (int)slot.size();
        c = create_ctx(p0.d, p0.n, p0.n_t, p0.n_c, p0.beta, p0.reg_type, p0.stokes, precision, 0, st, B);
        const long N1 = c->g.N1, N = c->N();
        const int K = c->n_c * c->d;
        c->betas.resize(B);
        for (int q = 0; q < B; ++q) c->betas[q] = problems[ids[slot[q]]].beta;
        REG_CUDA(cudaMemcpyAsync(c->betas_dev.get(B), c->betas.data(), B * sizeof(double), cudaMemcpyHostToDevice, st));
        double* mT = c->mT.get(N);
        double* mR = c->mR.get(N);
        double* v = c->sv_v.get(c->ncdN());
        for (int q = 0; q < B; ++q) {
          const reg_problem& p = problems[ids[slot[q]]];
          REG_CUDA(cudaMemcpyAsync(mT + q * N1, p.m_T, N1 * sizeof(double), cudaMemcpyDefault, st));
          REG_CUDA(cudaMemcpyAsync(mR + q * N1, p.m_R, N1 * sizeof(double), cudaMemcpyDefault, st));
          for (int k = 0; k < K; ++k)
            REG_CUDA(cudaMemcpyAsync(v + ((long)k * B + q) * N1, p.v + (long)k * N1, N1 * sizeof(double),
                                     cudaMemcpyDefault, st));
        }
        c->have_images = true;
        const bool more = solve_lockstep(c, v, o, S, slot, resume, kRestackMin);
        for (int q = 0; q < B; ++q) {  // iterates back to the callers' arrays (final for stopped problems)
          const reg_problem& p = problems[ids[slot[q]]];
          for (int k = 0; k < K; ++k)
            REG_CUDA(cudaMemcpyAsync(p.v + (long)k * N1, v + ((long)k * B + q) * N1, N1 * sizeof(double),
                                     cudaMemcpyDefault, st));
        }
        REG_CUDA(cudaStreamSynchronize(st));
        delete c;
        c = nullptr;
        if (!more) break;
        std::vector<int> live;
        for (int q : slot)
          if (S.active[q]) live.push_back(q);
        slot.swap(live);
        resume = true;
      }
      const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
      for (size_t q = 0; q < ids.size(); ++q) {
        S.R[q].seconds = secs;
        if (reports) reports[ids[q]] = S.R[q];
        if (S.R[q].status != REG_OK && S.R[q].status != REG_EMAXIT && status[si] == REG_OK) {
          status[si] = S.R[q].status;
          errors[si] = "problem " + std::to_string(ids[q]) + " ended with status " + std::to_string(S.R[q].status);
        }
      }
    } catch (const StatusError& e) {
      status[si] = e.status;
      errors[si] = e.what;
    } catch (const CudaError& e) {
      status[si] = e.code == cudaErrorMemoryAllocation ? REG_ENOMEM : REG_ECUDA;
      errors[si] = e.what;
    } catch (const std::bad_alloc&) {
      status[si] = REG_ENOMEM;
      errors[si] = "host allocation failed";
    }
    delete c;
    if (st) cudaStreamDestroy(st);
  };
  // the stacks run concurrently, one thread and stream each
  std::vector<std::thread> pool;
  for (size_t si = 0; si < stacks.size(); ++si) pool.emplace_back(run, si);
  for (auto& t : pool) t.join();
  for (size_t si = 0; si < stacks.size(); ++si)
    if (status[si] != REG_OK) {
      g_create_error = "reg_solve_lockstep: " + errors[si];
      return (reg_status)status[si];
    }
  return REG_OK;
}

reg_status reg_solve(reg_ctx* ctx, double* v_inout, const reg_solve_opts* opts, reg_solve_report* report) {
  API_BEGIN(ctx)
  reg_solve_opts o;
  reg_solve_opts_default(&o);
  if (opts) o = *opts;
  if (!v_inout) throw StatusError{REG_EINVAL, "v_inout is null"};
  Output io(c_, v_inout, c_->ncdN(), c_->stage_out);
  if (io.host)
    REG_CUDA(cudaMemcpyAsync(io.dev, v_inout, c_->ncdN() * sizeof(double), cudaMemcpyHostToDevice, c_->s));
  reg_solve_report R;
  int st = solve(c_, io.dev, o, R);
  io.finish();
  if (report) *report = R;
  if (st != REG_OK) throw StatusError{st, st == REG_EMAXIT ? "outer iteration cap reached" : "line search failed"};
  API_END
}

}  // extern "C"
