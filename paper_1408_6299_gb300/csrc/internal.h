// internal.h -- host-side declarations shared by the translation units of the
// registration library (not part of the public C ABI, see include/reg.h).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "fft.cuh"

namespace reg {

// CUDA error -> exception carrying the failing call, caught at the C ABI.
struct CudaError {
  cudaError_t code;
  std::string what;
};
struct StatusError {
  int status;
  std::string what;
};

#define REG_CUDA(call)                                                                      \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess) throw ::reg::CudaError{e_, std::string(#call) + ": " +           \
                                                      cudaGetErrorString(e_)};              \
  } while (0)
#define REG_LAUNCH()         \
  do {                       \
    ::reg::count_launch();   \
    REG_CUDA(cudaGetLastError()); \
  } while (0)

// ---------------------------------------------------------------------------
// Kernel accounting: a process-wide launch counter, and optional CUDA-event
// bracketing of launches by kind (enabled per context through the C ABI).
// ---------------------------------------------------------------------------
enum KernelKind {
  KK_ROWS_R2C = 0,  // real-to-complex row pass
  KK_ROWS_C2R = 1,  // complex-to-real row pass
  KK_COLS = 2,      // strided complex pass
  KK_MULT = 3,      // Fourier multipliers
  KK_STAGE = 4,     // Heun stage / transport right-hand side
  KK_FORCE = 5,     // body-force accumulation
  KK_OTHER = 6,     // everything else
  KK_COUNT = 7
};
void count_launch();
void add_launches(long n);  // kernels launched by a graph replay
long launch_count();

struct KernelProfiler {
  unsigned mask = 0;
  struct Rec {
    int kind;
    cudaEvent_t a, b;
    double bytes, flops;
  };
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
  double last_flops[KK_COUNT] = {0};  // per kind, of the last collected window
  ~KernelProfiler();
  cudaEvent_t take();
  void collect(double* ms, double* bytes, long* count);  // synchronises
};
extern thread_local KernelProfiler* tl_prof;

// bracket one launch; bytes = algorithmic bytes moved by it, flops = the
// floating-point operations of its transforms (0 where not counted)
struct ProfScope {
  int kind;
  cudaStream_t s;
  double bytes, flops;
  cudaEvent_t a = nullptr;
  ProfScope(int k, cudaStream_t st, double b, double f = 0.0);
  ~ProfScope();
};

// Periodic nodal grid, row-major with the last axis fastest. Real fields hold
// N values; packed half spectra hold Nc = N/2 complex values laid out as
// [n_0]..[n_{d-2}][M], M = n_{d-1}/2, where slot 0 of the last axis carries
// uhat(k',0) + i*uhat(k',n_{d-1}/2) (DC and Nyquist columns of the last axis).
// A grid of B independent problems of the same shape, stacked along an
// untransformed leading axis (B = 1: one problem). N, Nc and rows count all
// problems; every field is laid out [B][n_0]...[n_{d-1}].
struct Grid {
  int d = 0;
  int n[3] = {1, 1, 1};
  long N = 0;   // real points
  long Nc = 0;  // packed spectral points
  int L = 0;    // last-axis length
  int M = 0;    // L/2
  long rows = 0;  // N / L
  int B = 1;      // stacked problems
  long N1 = 0;    // real points of one problem
};

Grid make_grid(int d, const int64_t* n, int batch = 1);

// set the text that reg_last_error(NULL) returns on this thread
void set_thread_error(const std::string& msg);

// Persistent autotuner choices (tune.cu): -1 when the key has none yet.
// Keys start with tune_device_tag() (device name / multiprocessor count).
int tune_lookup(const std::string& key);
void tune_store(const std::string& key, int choice);
std::string tune_device_tag();

// Batched power-of-two FFTs and Fourier multipliers on one grid, in precision T.
template <typename T>
class Spectral {
 public:
  using C = cx<T>;
  Spectral(const Grid& g, cudaStream_t s);
  // Non-owning engine over device tables laid out as write_tables() lays out
  // its host image; allocates and copies nothing.
  Spectral(const Grid& g, cudaStream_t s, C* tables, const long* tw_off, long rc_off);
  ~Spectral();
  // Host image of the twiddle tables of every FFT length 4..512 followed by
  // the real-to-complex tables of every last-axis length 8..512 (double,
  // interleaved re/im). tw_off[e] / rc_off[e]: complex offset of the tables of
  // length 2^e. out may be null to query the size; returns complex entries.
  static long write_tables(double* out, long* tw_off, long* rc_off);
  Spectral(const Spectral&) = delete;
  Spectral& operator=(const Spectral&) = delete;

  const Grid& grid() const { return g_; }
  cudaStream_t stream() const { return s_; }

  // real field -> packed spectrum (unnormalised)
  void fwd(const T* u, C* U);
  // packed spectrum -> real field (normalised by 1/N); U is overwritten
  void inv(C* U, T* u);
  // G[i] = d/dx_i u, i < d  (first derivatives with the Nyquist mode dropped)
  void grad(const T* u, T* G, C* U, C* W);
  // out = sum_i d/dx_i q_i
  void div(const T* q, T* out, C* U, C* S);
  // W = i k~_axis U (W may equal U)
  void mult_deriv(const C* U, C* W, int axis);
  // S (+)= i k~_axis U
  void mult_deriv_acc(const C* U, C* S, int axis, bool first);
  // in place Leray projection of d spectra (stride Nc)
  void mult_leray(C* W);

  const C* twiddles(int L) const;   // Stockham stage tables for length L
  const C* rc_twiddles() const;     // exp(-2 pi i k / L_last), k < M
  // single precision, two-stage plans (L = 32..256): the stage-1 twiddle
  // block of length L with each entry (c, s) stored as (c, c, s, s), for the
  // paired column passes; null otherwise
  const float4* pair_twiddles(int L) const;

  // A second stream with a fork and a join event, for independent passes of
  // one stage (created on first use).
  cudaStream_t aux_stream();
  cudaEvent_t fork_event() const { return ev_fork_; }
  cudaEvent_t join_event() const { return ev_join_; }

 private:
  void cols(C* U, int axis, bool inverse);
  Grid g_;
  cudaStream_t s_;
  cudaStream_t aux_ = nullptr;
  cudaEvent_t ev_fork_ = nullptr, ev_join_ = nullptr;
  C* tw_ = nullptr;  // device: tables per length + real/complex table
  float4* tw2_ = nullptr;  // device: paired twiddle blocks (single precision only)
  long tw2_off_[11] = {0};
  bool owns_ = true;
  long tw_off_[11] = {0};  // offset of the table of length 2^e
  long rc_off_ = 0;
};

// ---------------------------------------------------------------------------
// Fused Heun stages (fused.cuh): advection k = -v.grad u [- grad m . v~] and
// divergence k = div(v lam), each with its Runge-Kutta update in the last pass.
// ---------------------------------------------------------------------------
// bounded waits of the TMA column pass that gave up since the last call
// (per precision; synchronises s)
int take_tma_timeouts_f32(cudaStream_t s);
int take_tma_timeouts_f64(cudaStream_t s);

namespace fused {
template <typename T>
struct AdvEpi;
template <typename T>
struct DivEpi;
}  // namespace fused
// three packed-spectrum scratch buffers per call (Zx unused in 2D). u_ready:
// U already holds the packed spectrum of u (no real-to-complex pass); emit:
// the last pass leaves the packed spectrum of the stage's out1 in U.
template <typename T>
void adv_stage(Spectral<T>& sp, const T* u, const fused::AdvEpi<T>& e, cx<T>* U, cx<T>* Zx, cx<T>* Zy,
               bool u_ready = false, bool emit = false);
// two 3D advection stages (fields uA, uB) sharing their passes; Z: six
// spectral work arrays of Nc values
template <typename T>
void adv2_stage(Spectral<T>& sp, const T* uA, const fused::AdvEpi<T>& eA, const T* uB, const fused::AdvEpi<T>& eB,
                cx<T>* const* Z);
// a: d velocity fields at stride N
template <typename T>
void div_stage(Spectral<T>& sp, const T* lam, const T* a, const fused::DivEpi<T>& e, cx<T>* Q0, cx<T>* Q1, cx<T>* Q2);

// ---------------------------------------------------------------------------
// Fourier-diagonal operators on whole coefficient vectors (FP64), with the
// DC/Nyquist pairing of the packed last-axis slot 0.
// ---------------------------------------------------------------------------
// out_l = beta sum_l' Cg[l][l'] a(k) V_l' + (stokes ? K F_l : F_l); F may be null.
// betas (device, may be null): one beta per stacked problem, replacing beta.
void spec_tail(const Grid& g, cudaStream_t s, const double2* V, const double2* F, double2* out, int nc,
               double beta, const double* Cg_dev, int reg, int stokes, const double* betas = nullptr);
// out_l = sum_l' Ci[l][l'] s(k) R_l' with s = 1/(beta a(k)), s = 1 at k = 0.
void spec_precond(const Grid& g, cudaStream_t s, const double2* R, double2* out, int nc, double beta,
                  const double* Ci_dev, int reg, const double* betas = nullptr);
// Gaussian filter exp(-sigma^2 |k|^2 / 2) of one packed FP64 field (out may not alias U)
void spec_gauss(const Grid& g, cudaStream_t s, double2* U, double2* out, double sigma);
// trigonometric interpolation of nfields packed FP64 spectra of grid c onto the
// finer grid f (every axis refined by a factor >= 2; one problem, no stacking)
void spec_upsample(const Grid& c, const Grid& f, cudaStream_t s, const double2* P, double2* Q, int nfields);

}  // namespace reg
