// pointwise.h -- launchers of the pointwise transport stages, vector kernels
// and deterministic FP64 reductions (pointwise.cu).
#pragma once
#include "internal.h"

namespace reg {

// small coefficient table passed by value (Chebyshev values, quadrature weights)
struct Coefs {
  double c[16];
};

// out[x] = sum_l b_l coef[l*dN + x], x < dN
template <typename T, typename S>
void vel_at(const S* coef, int nc, const Coefs& b, T* out, long dN, cudaStream_t s);
template <typename S, typename T>
void convert(const S* in, T* out, long n, cudaStream_t s);

// Heun stage 1 of m' = -v.G - gm.w (the gm.w source only when gm != null; G may
// be null for a zero state; y may be null for a zero state):
//   yh = y + h k, acc = y + h/2 k.
template <typename T>
void transport_stage1(const T* G, const T* vt, const T* gm, const T* wt, const T* y, T h, T* yh, T* acc, int d,
                      long N, cudaStream_t s);
// out = sum_i a_i b_i (d fields at stride N)
template <typename T>
void dot_fields(const T* a, const T* b, T* out, int d, long N, cudaStream_t s);
// f[l][i] += c_l lam gm_i: plain sum into fhi (flo null) or a compensated
// (fhi, flo) pair of precision T
template <typename T>
void force_acc(T* fhi, T* flo, const T* lam, const T* gm, const Coefs& c, int nc, int d, long N, cudaStream_t s);
// out = (double)hi + (double)lo
void pair_to_double(const float* hi, const float* lo, double* out, long n, cudaStream_t s);

void detF_rhs(const double* G, const double* vt, const double* gv, const double* F, int q, double* k, int d, long N,
              cudaStream_t s);
void identity_tensor(double* F, int d, long N, cudaStream_t s);
void det_tensor(const double* F, double* det, int d, long N, cudaStream_t s);
// smallest acute angle between deformed grid edges (columns of F) per point
void grid_angle_tensor(const double* F, double* angle, int d, long N, cudaStream_t s);

// out = a x + b y in precision T (y may be null: out = a x; out may alias x or y)
template <typename T>
void lincomb_t(T a, const T* x, T b, const T* y, T* out, long n, cudaStream_t s);

// y = a x + b y ; out = a x + b y
void axpby(double a, const double* x, double b, double* y, long n, cudaStream_t s);
void lincomb(double a, const double* x, double b, const double* y, double* out, long n, cudaStream_t s);

// reductions (synchronise the stream; scratch holds reduce_scratch_doubles())
long reduce_scratch_doubles();
double dot(const double* a, const double* b, long n, double* scratch, cudaStream_t s);
double sqdiff(const double* a, const double* b, long n, double* scratch, cudaStream_t s);
double maxabs(const double* a, long n, double* scratch, cudaStream_t s);
void stats(const double* a, long n, double* scratch, cudaStream_t s, double out[4]);

// per-problem reductions of B stacked problems, vectors of K components laid
// out [K][B][N1]; results (B values) to host memory; scratch holds
// seg_scratch_doubles(B); synchronise the stream
long seg_scratch_doubles(int B);
void seg_dot(const double* a, const double* b, int K, int B, long N1, double* scratch, cudaStream_t s, double* out);
void seg_sqdiff(const double* a, const double* b, int K, int B, long N1, double* scratch, cudaStream_t s,
                double* out);
void seg_maxabs(const double* a, int K, int B, long N1, double* scratch, cudaStream_t s, double* out);
// out = a_p x + c_p y per problem p; a_dev, c_dev: B coefficients on the device (out may alias y)
void lincomb_seg(const double* a_dev, const double* x, const double* c_dev, const double* y, double* out, int K,
                 int B, long N1, cudaStream_t s);
// the same reductions with the B results left in device memory (no synchronisation;
// usable inside a captured graph)
void seg_dot_dev(const double* a, const double* b, int K, int B, long N1, double* scratch, cudaStream_t s,
                 double* out_dev);
void seg_sqdiff_dev(const double* a, const double* b, int K, int B, long N1, double* scratch, cudaStream_t s,
                    double* out_dev);

// ---------------------------------------------------------------------------
// Per-problem scalars of the device-driven lockstep loops (PCG, Nocedal &
// Wright Alg. 5.3, with the forcing term of Eq. termination-criterion-ksm;
// Armijo backtracking, Sec. 3.2): rows of B doubles in one array lk, and an
// int control block ctl. Every decision a problem takes is the host loop's,
// in the same floating-point operations (no contraction), so a problem follows
// the same iterates either way.
// ---------------------------------------------------------------------------
enum LockSlot {
  LK_ACT = 0,   // problem still iterating (1/0)
  LK_ON,        // PCG still running for the problem
  LK_ETA,       // forcing term
  LK_G2,        // ||g||_2
  LK_G02,       // ||g_0||_2
  LK_RZ, LK_RZN, LK_RN2, LK_PHP,
  LK_A,         // PCG step length (0 for problems not running)
  LK_NEGC,      // 1: copy p into s (negative curvature at the first PCG step)
  LK_KEEP,      // 1 - LK_NEGC
  LK_MZ, LK_BT, // coefficients of p = mz z + bt p
  LK_ONE, LK_ZERO, LK_MONE,
  LK_J,         // objective at the iterate
  LK_JT,        // trial objective
  LK_SLOPE,     // <g, s>_h
  LK_ALPHA,     // line-search step length
  LK_SRCH,      // line search still running
  LK_D2, LK_R2, // distance and regularisation sums of the trial point (unscaled)
  LK_PCG, LK_MV, LK_NPDE, LK_LS,  // counters added to the reports
  LK_STATUS,    // reg_status set on the device (0: none)
  LK_COUNT
};
enum LockCtl { LC_IT = 0, LC_PIT, LC_LST, LC_ON, LC_COUNT };
// constants and counters reset; LK_ON = LK_ACT, LK_ETA = min(0.5, sqrt(g2 / g02)); ctl zeroed
void lk_pcg_init(double* lk, int* ctl, int B, cudaStream_t s);
// top of a PCG iteration (after rn2 = <r, r>): stop the problems that reached
// the forcing term; sets the IF handle (some problem runs and fewer than
// maxit iterations ran in this PCG solve) and the WHILE handle (the same, and
// fewer than cap iterations ran in this launch)
void lk_pcg_check(double* lk, int* ctl, int B, int cap, int maxit, unsigned long long h_if,
                  unsigned long long h_while, cudaStream_t s);
// after pHp = <p, H p>: step lengths, curvature guard, counters
void lk_pcg_alpha(double* lk, int* ctl, int B, cudaStream_t s);
// after rzn = <r, z>: coefficients of the new direction
void lk_pcg_beta(double* lk, int* ctl, int B, cudaStream_t s);
// line search: slope *= h_d; alpha = 1 and search for active problems
void lk_ls_init(double* lk, int* ctl, int B, double hd, cudaStream_t s);
// top of a trial: IF handle (some problem searches), WHILE handle (and fewer than max_bt trials)
void lk_ls_check(double* lk, int* ctl, int B, int max_bt, unsigned long long h_if, unsigned long long h_while,
                 cudaStream_t s);
// after the trial objective (LK_D2, LK_R2): Armijo test, backtracking
void lk_ls_armijo(double* lk, int B, double hd, double c1, double rho, cudaStream_t s);
// problems still searching fail (REG_ELINESEARCH); stopped problems take no step
void lk_ls_final(double* lk, int B, int status_ls, cudaStream_t s);

}  // namespace reg
