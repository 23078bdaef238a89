/*
 * oracle.c -- plain, slow, double-precision CPU reference for the inexact
 * Gauss-Newton-Krylov image registration method of Mang & Biros,
 * "An inexact Newton-Krylov algorithm for constrained diffeomorphic image
 * registration" (arXiv:1408.6299).
 *
 * TEST INFRASTRUCTURE. Only the test suite, the package's smoke check and the
 * CPU-baseline leg of the benchmark load this library. The CUDA library never
 * calls it, and the two share no source, header, table or helper.
 *
 * Conventions (every function below follows them):
 *   - grid: d in {2,3}, sizes n[0..d-1] (powers of two), row-major with the
 *     last axis fastest; N = prod n. Nodes x_j = 2*pi*j/n_i (Sec. 3.3.1; the
 *     periodic shift of the paper's (-pi,pi)^d is immaterial).
 *   - time: h_t = 1/n_t, t_j = j*h_t, j = 0..n_t (Sec. 3.3.1).
 *   - velocity coefficients v[l][i][x], l < n_c (Chebyshev index), i < d
 *     (Eq. expansion, Sec. 3.3.2).
 *   - all arithmetic is IEEE double, no fused multiply-add contraction
 *     (compiled with -ffp-contract=off) so results agree across machines.
 *
 * Readings of passages the paper leaves open (each is stated where it is used):
 *   R1 Nyquist: first derivatives and the Leray projection use the masked
 *      wavenumber (k_i = -n_i/2 replaced by 0); the regularisation symbol
 *      a(k) keeps the full k (pinned by the beta=1e6 eigenvalues, Tab. 5.2).
 *   R2 RK2 is Heun's method (explicit trapezoid), Sec. 3.3.1.
 *   R3 Chebyshev Gram matrix is the exact integral over [0,1] (App. A).
 *   R4 Time quadrature of the body force is the trapezoid rule
 *      (optimize-then-discretize, Sec. 3); a discrete-adjoint variant is kept
 *      for tests only.
 */
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENOMEM 2
#define ORC_ECFL 6
#define ORC_ELINESEARCH 7
#define ORC_EMAXIT 8

typedef struct {
  int d;         /* space dimension, 2 or 3 */
  int n[3];      /* grid points per axis (last axis fastest) */
  int n_t;       /* number of RK2 time steps */
  int n_c;       /* number of Chebyshev coefficient fields in time */
  double beta;   /* regularisation weight */
  int reg;       /* 1: H1 seminorm (A = -Lap), 2: H2 seminorm (A = Lap^2) */
  int stokes;    /* 1: Leray-project the body force (gamma = 1) */
  int dto;       /* 0: trapezoid quadrature (paper); 1: discrete adjoint */
} orc_prob;

typedef struct {
  double grad_rtol;      /* stop when ||g||_inf / ||g_0||_inf <= grad_rtol */
  int max_outer;         /* outer iteration cap (n_opt) */
  double armijo_c1;      /* sufficient-decrease constant */
  double backtrack;      /* step reduction factor */
  int max_backtracks;    /* line-search trials */
  int pcg_maxit;         /* 0: use n (order of the reduced system) */
  int newton;            /* 1: full Newton Hessian in PCG (N-PCG), else Gauss-Newton */
  int picard;            /* 1: Picard / preconditioned gradient descent (Eq. picard) instead of PCG */
  int step_memory;       /* 1: Picard step memory alpha~ (Sec. 3.3.5) */
  int stop_rule;         /* 0: relative gradient; 1: the C1-C5 set (Eq. stopping-criteria) */
  double tau_J;          /* tolerance of C1-C3 */
  double cfl_max;        /* > 0: halve the step while CFL(v + s) exceeds it */
} orc_opts;

typedef struct {
  int outer;          /* outer iterations taken */
  int pcg_iters;      /* total PCG iterations */
  int matvecs;        /* Hessian applications */
  int n_pde;          /* hyperbolic PDE solves (Sec. 5.2 measure) */
  int ls_trials;      /* objective evaluations inside line searches */
  int status;         /* ORC_OK or error code */
  double J0, J;       /* first and final objective */
  double g0_inf, g_inf;
  double g0_2, g_2;
  int stop_flags;     /* bit i-1: criterion Ci held at exit (stop_rule 1) */
  int cfl_halvings;   /* step halvings forced by cfl_max */
  double alpha_mem;   /* final Picard step memory alpha~ */
  double J_prev;      /* objective of the previous iterate */
  double dv_inf;      /* ||v_{k-1} - v_k||_inf of the last step */
  double v_inf;       /* ||v_k||_inf */
} orc_report;

/* ------------------------------------------------------------------ */
/* small helpers                                                       */
/* ------------------------------------------------------------------ */

static long grid_N(const orc_prob *P) {
  long N = 1;
  for (int i = 0; i < P->d; ++i) N *= P->n[i];
  return N;
}

static int is_pow2(int n) { return n >= 2 && (n & (n - 1)) == 0; }

static int prob_ok(const orc_prob *P) {
  if (P->d != 2 && P->d != 3) return 0;
  for (int i = 0; i < P->d; ++i)
    if (!is_pow2(P->n[i])) return 0;
  if (P->n_t < 1 || P->n_c < 1 || !(P->beta >= 0.0)) return 0;
  if (P->reg != 1 && P->reg != 2) return 0;
  return 1;
}

/* full signed wavenumber of index j on an axis of n points:
 * 0..n/2-1 -> j, n/2..n-1 -> j-n (so j = n/2 maps to -n/2). */
static double wavenumber(int j, int n) { return (j < n / 2) ? (double)j : (double)(j - n); }

/* masked first-derivative wavenumber (reading R1): Nyquist -> 0 */
static double wavenumber_masked(int j, int n) { return (j == n / 2) ? 0.0 : wavenumber(j, n); }

/* per-axis index of flat index idx */
static void unflatten(const orc_prob *P, long idx, int *j) {
  for (int i = P->d - 1; i >= 0; --i) {
    j[i] = (int)(idx % P->n[i]);
    idx /= P->n[i];
  }
}

/* ------------------------------------------------------------------ */
/* FFT: iterative radix-2 Cooley-Tukey on complex doubles (re, im      */
/* interleaved). Forward is unnormalised, exp(-2 pi i jk/n); inverse   */
/* uses exp(+2 pi i jk/n) and divides by n per axis (1/N in total).    */
/* ------------------------------------------------------------------ */

static void fft1d(double *a, int n, int inverse, const double *cs, const double *sn) {
  /* bit-reversal permutation */
  for (int i = 1, j = 0; i < n; ++i) {
    int bit = n >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) {
      double tr = a[2 * i], ti = a[2 * i + 1];
      a[2 * i] = a[2 * j];
      a[2 * i + 1] = a[2 * j + 1];
      a[2 * j] = tr;
      a[2 * j + 1] = ti;
    }
  }
  /* butterflies; cs[k] + i*sn[k] = exp(-2 pi i k / n) */
  for (int len = 2; len <= n; len <<= 1) {
    int half = len / 2, step = n / len;
    for (int s = 0; s < n; s += len) {
      for (int k = 0; k < half; ++k) {
        double wr = cs[k * step];
        double wi = inverse ? -sn[k * step] : sn[k * step];
        double *u = a + 2 * (s + k), *w = a + 2 * (s + k + half);
        double tr = wr * w[0] - wi * w[1];
        double ti = wr * w[1] + wi * w[0];
        w[0] = u[0] - tr;
        w[1] = u[1] - ti;
        u[0] = u[0] + tr;
        u[1] = u[1] + ti;
      }
    }
  }
  if (inverse) {
    double s = 1.0 / n;
    for (int i = 0; i < 2 * n; ++i) a[i] *= s;
  }
}

/* In-place d-dimensional complex FFT of N complex values. */
int orc_fft(int d, const int *n, double *data, int inverse) {
  long N = 1;
  for (int i = 0; i < d; ++i) {
    if (!is_pow2(n[i]) && n[i] != 1) return ORC_EINVAL;
    N *= n[i];
  }
  for (int ax = 0; ax < d; ++ax) {
    int L = n[ax];
    if (L == 1) continue;
    long stride = 1;
    for (int i = ax + 1; i < d; ++i) stride *= n[i];
    long npencil = N / L;
    double *cs = malloc(sizeof(double) * L), *sn = malloc(sizeof(double) * L);
    if (!cs || !sn) { free(cs); free(sn); return ORC_ENOMEM; }
    for (int k = 0; k < L; ++k) {
      double ang = -2.0 * M_PI * (double)k / (double)L;
      cs[k] = cos(ang);
      sn[k] = sin(ang);
    }
    int fail = 0;
#pragma omp parallel
    {
      double *buf = malloc(sizeof(double) * 2 * L);
      if (!buf) {
#pragma omp atomic write
        fail = 1;
      } else {
#pragma omp for schedule(static)
        for (long p = 0; p < npencil; ++p) {
          long outer = p / stride, inner = p % stride;
          long base = outer * L * stride + inner;
          for (int j = 0; j < L; ++j) {
            buf[2 * j] = data[2 * (base + j * stride)];
            buf[2 * j + 1] = data[2 * (base + j * stride) + 1];
          }
          fft1d(buf, L, inverse, cs, sn);
          for (int j = 0; j < L; ++j) {
            data[2 * (base + j * stride)] = buf[2 * j];
            data[2 * (base + j * stride) + 1] = buf[2 * j + 1];
          }
        }
        free(buf);
      }
    }
    free(cs);
    free(sn);
    if (fail) return ORC_ENOMEM;
  }
  return ORC_OK;
}

/* real field -> complex spectrum (imaginary part zero before the transform) */
static int to_spectrum(const orc_prob *P, const double *u, double *U) {
  long N = grid_N(P);
#pragma omp parallel for schedule(static)
  for (long x = 0; x < N; ++x) {
    U[2 * x] = u[x];
    U[2 * x + 1] = 0.0;
  }
  return orc_fft(P->d, P->n, U, 0);
}

/* complex spectrum -> real part of the inverse transform */
static int from_spectrum(const orc_prob *P, double *U, double *u) {
  int st = orc_fft(P->d, P->n, U, 1);
  if (st) return st;
  long N = grid_N(P);
#pragma omp parallel for schedule(static)
  for (long x = 0; x < N; ++x) u[x] = U[2 * x];
  return ORC_OK;
}

/* regularisation symbol a(k) = |k|^2 (H1) or |k|^4 (H2), full k (R1). */
static double reg_symbol(const orc_prob *P, const int *j) {
  double kk = 0.0;
  for (int i = 0; i < P->d; ++i) {
    double k = wavenumber(j[i], P->n[i]);
    kk += k * k;
  }
  return P->reg == 1 ? kk : kk * kk;
}

/* ------------------------------------------------------------------ */
/* Spectral operators (Sec. 3.3.1 Fourier collocation; Sec. 3.3.3;      */
/* Sec. 3.3.4 / App. B for the Leray projection K).                    */
/* ------------------------------------------------------------------ */

/* out[i] = d/dx_i u  (i < d), each N reals: Re F^{-1}[ i k~_i F u ] */
int orc_grad(const orc_prob *P, const double *u, double *out) {
  long N = grid_N(P);
  double *U = malloc(sizeof(double) * 2 * N), *W = malloc(sizeof(double) * 2 * N);
  if (!U || !W) { free(U); free(W); return ORC_ENOMEM; }
  int st = to_spectrum(P, u, U);
  for (int i = 0; i < P->d && !st; ++i) {
#pragma omp parallel for schedule(static)
    for (long x = 0; x < N; ++x) {
      int j[3];
      unflatten(P, x, j);
      double k = wavenumber_masked(j[i], P->n[i]);
      /* (i k) * (a + i b) = -k b + i k a */
      W[2 * x] = -k * U[2 * x + 1];
      W[2 * x + 1] = k * U[2 * x];
    }
    st = from_spectrum(P, W, out + i * N);
  }
  free(U);
  free(W);
  return st;
}

/* out = div w = sum_i d/dx_i w_i */
int orc_div(const orc_prob *P, const double *w, double *out) {
  long N = grid_N(P);
  double *U = malloc(sizeof(double) * 2 * N), *S = calloc(2 * N, sizeof(double));
  if (!U || !S) { free(U); free(S); return ORC_ENOMEM; }
  int st = 0;
  for (int i = 0; i < P->d && !st; ++i) {
    st = to_spectrum(P, w + i * N, U);
    if (st) break;
#pragma omp parallel for schedule(static)
    for (long x = 0; x < N; ++x) {
      int j[3];
      unflatten(P, x, j);
      double k = wavenumber_masked(j[i], P->n[i]);
      S[2 * x] += -k * U[2 * x + 1];
      S[2 * x + 1] += k * U[2 * x];
    }
  }
  if (!st) st = from_spectrum(P, S, out);
  free(U);
  free(S);
  return st;
}

/* out = A u for one scalar field: F^{-1}[a(k) F u] (Eq. first-variation-H1/H2) */
int orc_apply_A(const orc_prob *P, const double *u, double *out) {
  long N = grid_N(P);
  double *U = malloc(sizeof(double) * 2 * N);
  if (!U) return ORC_ENOMEM;
  int st = to_spectrum(P, u, U);
  if (!st) {
#pragma omp parallel for schedule(static)
    for (long x = 0; x < N; ++x) {
      int j[3];
      unflatten(P, x, j);
      double a = reg_symbol(P, j);
      U[2 * x] *= a;
      U[2 * x + 1] *= a;
    }
    st = from_spectrum(P, U, out);
  }
  free(U);
  return st;
}

/* out = K w = w - grad Lap^{-1} div w (Eq. eliminated-control), per mode
 * (I - k~ k~^T / |k~|^2) with the identity where |k~| = 0. w, out: d fields. */
int orc_leray(const orc_prob *P, const double *w, double *out) {
  long N = grid_N(P);
  int d = P->d;
  double *U = malloc(sizeof(double) * 2 * N * d);
  if (!U) return ORC_ENOMEM;
  int st = 0;
  for (int i = 0; i < d && !st; ++i) st = to_spectrum(P, w + i * N, U + 2 * i * N);
  if (!st) {
#pragma omp parallel for schedule(static)
    for (long x = 0; x < N; ++x) {
      int j[3];
      double k[3];
      unflatten(P, x, j);
      double kk = 0.0;
      for (int i = 0; i < d; ++i) {
        k[i] = wavenumber_masked(j[i], P->n[i]);
        kk += k[i] * k[i];
      }
      if (kk == 0.0) continue;
      double dr = 0.0, di = 0.0;
      for (int i = 0; i < d; ++i) {
        dr += k[i] * U[2 * (i * N + x)];
        di += k[i] * U[2 * (i * N + x) + 1];
      }
      for (int i = 0; i < d; ++i) {
        U[2 * (i * N + x)] -= k[i] * dr / kk;
        U[2 * (i * N + x) + 1] -= k[i] * di / kk;
      }
    }
    for (int i = 0; i < d && !st; ++i) st = from_spectrum(P, U + 2 * i * N, out + i * N);
  }
  free(U);
  return st;
}

/* ------------------------------------------------------------------ */
/* Chebyshev basis in time (Eq. expansion; App. A)                     */
/* ------------------------------------------------------------------ */

/* b_l(t) = T_l(2t - 1), l = 0..n_c-1 (0-based) */
void orc_cheb_eval(int n_c, double t, double *b) {
  double x = 2.0 * t - 1.0;
  for (int l = 0; l < n_c; ++l) {
    if (l == 0) b[l] = 1.0;
    else if (l == 1) b[l] = x;
    else b[l] = 2.0 * x * b[l - 1] - b[l - 2];
  }
}

/* integral of T_m over [-1,1]: 2/(1-m^2) for even m, 0 for odd m */
static double cheb_integral(int m) { return (m % 2) ? 0.0 : 2.0 / (1.0 - (double)m * m); }

/* C[l][l'] = int_0^1 b_l b_l' dt (reading R3: exact integral; App. A claims
 * orthogonality, which does not hold for this inner product). Uses
 * T_a T_b = (T_{a+b} + T_{|a-b|})/2 and dt = dx/2. */
void orc_cheb_gram(int n_c, double *C) {
  for (int a = 0; a < n_c; ++a)
    for (int b = 0; b < n_c; ++b)
      C[a * n_c + b] = 0.25 * (cheb_integral(a + b) + cheb_integral(abs(a - b)));
}

/* v(t) = sum_l b_l(t) v_l  (d fields) */
static void velocity_at(const orc_prob *P, const double *v, double t, double *vt) {
  long N = grid_N(P);
  int d = P->d, nc = P->n_c;
  double b[64];
  orc_cheb_eval(nc, t, b);
#pragma omp parallel for schedule(static)
  for (long x = 0; x < N; ++x)
    for (int i = 0; i < d; ++i) {
      double s = 0.0;
      for (int l = 0; l < nc; ++l) s += b[l] * v[((long)l * d + i) * N + x];
      vt[i * N + x] = s;
    }
}

/* ------------------------------------------------------------------ */
/* Transport operators                                                 */
/* ------------------------------------------------------------------ */

/* out = L m = -v . grad m  (right-hand side of Eq. first-order-forward) */
static int apply_L(const orc_prob *P, const double *vt, const double *m, double *out, double *gtmp) {
  long N = grid_N(P);
  int st = orc_grad(P, m, gtmp);
  if (st) return st;
#pragma omp parallel for schedule(static)
  for (long x = 0; x < N; ++x) {
    double s = 0.0;
    for (int i = 0; i < P->d; ++i) s += vt[i * N + x] * gtmp[i * N + x];
    out[x] = -s;
  }
  return ORC_OK;
}

/* out = D lam = div(v lam)  (Eq. first-order-adjoint, backward in time) */
static int apply_D(const orc_prob *P, const double *vt, const double *lam, double *out, double *wtmp) {
  long N = grid_N(P);
#pragma omp parallel for schedule(static)
  for (long x = 0; x < N; ++x)
    for (int i = 0; i < P->d; ++i) wtmp[i * N + x] = vt[i * N + x] * lam[x];
  return orc_div(P, wtmp, out);
}

/* State equation (Eq. first-order-forward), Heun steps forward in time:
 *   k1 = L(t_j) m_j, mh = m_j + h k1, k2 = L(t_{j+1}) mh,
 *   m_{j+1} = m_j + h/2 (k1 + k2).
 * mtraj: (n_t+1) x N. mhat (may be NULL): stage-2 inputs mh of step j stored
 * at slot j+1 (slot 0 unused). */
int orc_state(const orc_prob *P, const double *v, const double *m0, double *mtraj, double *mhat) {
  if (!prob_ok(P)) return ORC_EINVAL;
  long N = grid_N(P);
  int d = P->d, nt = P->n_t;
  double h = 1.0 / nt;
  double *va = malloc(sizeof(double) * d * N), *vb = malloc(sizeof(double) * d * N);
  double *k1 = malloc(sizeof(double) * N), *k2 = malloc(sizeof(double) * N);
  double *mh = malloc(sizeof(double) * N), *g = malloc(sizeof(double) * d * N);
  int st = (!va || !vb || !k1 || !k2 || !mh || !g) ? ORC_ENOMEM : ORC_OK;
  if (!st) memcpy(mtraj, m0, sizeof(double) * N);
  for (int j = 0; j < nt && !st; ++j) {
    const double *mj = mtraj + (long)j * N;
    double *mn = mtraj + (long)(j + 1) * N;
    velocity_at(P, v, j * h, va);
    velocity_at(P, v, (j + 1) * h, vb);
    st = apply_L(P, va, mj, k1, g);
    if (st) break;
#pragma omp parallel for schedule(static)
    for (long x = 0; x < N; ++x) mh[x] = mj[x] + h * k1[x];
    if (mhat) memcpy(mhat + (long)(j + 1) * N, mh, sizeof(double) * N);
    st = apply_L(P, vb, mh, k2, g);
    if (st) break;
#pragma omp parallel for schedule(static)
    for (long x = 0; x < N; ++x) mn[x] = mj[x] + 0.5 * h * (k1[x] + k2[x]);
  }
  free(va); free(vb); free(k1); free(k2); free(mh); free(g);
  return st;
}

/* Adjoint equation (Eq. first-order-adjoint) backward in time from lam_{n_t}:
 *   k1 = D(t_{j+1}) lam_{j+1}, lh = lam_{j+1} + h k1, k2 = D(t_j) lh,
 *   lam_j = lam_{j+1} + h/2 (k1 + k2).
 * This step is the exact transpose of the forward Heun step (L^T = D).
 * ltraj: (n_t+1) x N with ltraj[n_t] = lam_end. lhat (may be NULL): lh of the
 * step ending at j stored at slot j (slot n_t unused). */
int orc_adjoint(const orc_prob *P, const double *v, const double *lam_end, double *ltraj, double *lhat) {
  if (!prob_ok(P)) return ORC_EINVAL;
  long N = grid_N(P);
  int d = P->d, nt = P->n_t;
  double h = 1.0 / nt;
  double *va = malloc(sizeof(double) * d * N), *vb = malloc(sizeof(double) * d * N);
  double *k1 = malloc(sizeof(double) * N), *k2 = malloc(sizeof(double) * N);
  double *lh = malloc(sizeof(double) * N), *w = malloc(sizeof(double) * d * N);
  int st = (!va || !vb || !k1 || !k2 || !lh || !w) ? ORC_ENOMEM : ORC_OK;
  if (!st) memcpy(ltraj + (long)nt * N, lam_end, sizeof(double) * N);
  for (int j = nt - 1; j >= 0 && !st; --j) {
    const double *lj1 = ltraj + (long)(j + 1) * N;
    double *lj = ltraj + (long)j * N;
    velocity_at(P, v, (j + 1) * h, vb);
    velocity_at(P, v, j * h, va);
    st = apply_D(P, vb, lj1, k1, w);
    if (st) break;
#pragma omp parallel for schedule(static)
    for (long x = 0; x < N; ++x) lh[x] = lj1[x] + h * k1[x];
    if (lhat) memcpy(lhat + (long)j * N, lh, sizeof(double) * N);
    st = apply_D(P, va, lh, k2, w);
    if (st) break;
#pragma omp parallel for schedule(static)
    for (long x = 0; x < N; ++x) lj[x] = lj1[x] + 0.5 * h * (k1[x] + k2[x]);
  }
  free(va); free(vb); free(k1); free(k2); free(lh); free(w);
  return st;
}

/* ------------------------------------------------------------------ */
/* Regularisation and preconditioner on coefficient vectors            */
/* (n_c x d x N); App. A Eq. control-equation-expansion; Sec. 3.3.3.   */
/* ------------------------------------------------------------------ */

/* out_l = beta * sum_l' C_ll' A v_l'  */
int orc_reg_apply(const orc_prob *P, const double *v, double *out) {
  long N = grid_N(P);
  int d = P->d, nc = P->n_c;
  double C[64 * 64];
  orc_cheb_gram(nc, C);
  double *Av = malloc(sizeof(double) * (long)nc * d * N);
  if (!Av) return ORC_ENOMEM;
  int st = 0;
  for (long f = 0; f < (long)nc * d && !st; ++f) st = orc_apply_A(P, v + f * N, Av + f * N);
  if (!st) {
#pragma omp parallel for schedule(static)
    for (long x = 0; x < N; ++x)
      for (int l = 0; l < nc; ++l)
        for (int i = 0; i < d; ++i) {
          double s = 0.0;
          for (int m = 0; m < nc; ++m) s += C[l * nc + m] * Av[((long)m * d + i) * N + x];
          out[((long)l * d + i) * N + x] = P->beta * s;
        }
  }
  free(Av);
  return st;
}

/* invert a small SPD matrix by Gauss-Jordan with partial pivoting */
static int small_inverse(int n, const double *A, double *Ainv) {
  double M[64 * 128];
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < 2 * n; ++c) M[r * 2 * n + c] = (c < n) ? A[r * n + c] : (c - n == r ? 1.0 : 0.0);
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (fabs(M[r * 2 * n + c]) > fabs(M[piv * 2 * n + c])) piv = r;
    if (M[piv * 2 * n + c] == 0.0) return ORC_EINVAL;
    if (piv != c)
      for (int k = 0; k < 2 * n; ++k) {
        double t = M[c * 2 * n + k];
        M[c * 2 * n + k] = M[piv * 2 * n + k];
        M[piv * 2 * n + k] = t;
      }
    double p = M[c * 2 * n + c];
    for (int k = 0; k < 2 * n; ++k) M[c * 2 * n + k] /= p;
    for (int r = 0; r < n; ++r)
      if (r != c) {
        double f = M[r * 2 * n + c];
        for (int k = 0; k < 2 * n; ++k) M[r * 2 * n + k] -= f * M[c * 2 * n + k];
      }
  }
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < n; ++c) Ainv[r * n + c] = M[r * 2 * n + n + c];
  return ORC_OK;
}

/* z = P^{-1} r with P = beta C (x) A (Sec. 3.3.3): per Fourier mode
 * z^_l = sum_l' (C^{-1})_ll' r^_l' / (beta a(k)); on the k = 0 mode the
 * scaling 1/(beta a) is replaced by one, so there z^_l = sum (C^{-1})_ll' r^_l'. */
int orc_precond(const orc_prob *P, const double *r, double *z) {
  long N = grid_N(P);
  int d = P->d, nc = P->n_c;
  double C[64 * 64], Ci[64 * 64];
  orc_cheb_gram(nc, C);
  if (small_inverse(nc, C, Ci)) return ORC_EINVAL;
  double *R = malloc(sizeof(double) * 2 * (long)nc * d * N);
  double *Z = malloc(sizeof(double) * 2 * (long)nc * d * N);
  if (!R || !Z) { free(R); free(Z); return ORC_ENOMEM; }
  int st = 0;
  for (long f = 0; f < (long)nc * d && !st; ++f) st = to_spectrum(P, r + f * N, R + 2 * f * N);
  if (!st) {
#pragma omp parallel for schedule(static)
    for (long x = 0; x < N; ++x) {
      int j[3];
      unflatten(P, x, j);
      double a = reg_symbol(P, j);
      double s = (x == 0) ? 1.0 : 1.0 / (P->beta * a);
      for (int l = 0; l < nc; ++l)
        for (int i = 0; i < d; ++i) {
          double zr = 0.0, zi = 0.0;
          for (int m = 0; m < nc; ++m) {
            zr += Ci[l * nc + m] * R[2 * (((long)m * d + i) * N + x)];
            zi += Ci[l * nc + m] * R[2 * (((long)m * d + i) * N + x) + 1];
          }
          Z[2 * (((long)l * d + i) * N + x)] = s * zr;
          Z[2 * (((long)l * d + i) * N + x) + 1] = s * zi;
        }
    }
    for (long f = 0; f < (long)nc * d && !st; ++f) st = from_spectrum(P, Z + 2 * f * N, z + f * N);
  }
  free(R);
  free(Z);
  return st;
}

/* ------------------------------------------------------------------ */
/* Objective, gradient, Gauss-Newton Hessian matvec                    */
/* ------------------------------------------------------------------ */

static double cell_volume(const orc_prob *P) {
  double h = 1.0;
  for (int i = 0; i < P->d; ++i) h *= 2.0 * M_PI / P->n[i];
  return h;
}

/* J = 1/2 ||m_R - m_1||^2_h + beta/2 sum_ll' C_ll' <B v_l, B v_l'>_h
 * (Eq. objective with the expansion of App. A Eq. regularization-expansion),
 * <u, w>_h = h_d sum_x u w and <Bu, Bw> = <u, A w>.
 * out[0] = J, out[1] = distance term, out[2] = regularisation term. */
int orc_objective(const orc_prob *P, const double *v, const double *mT, const double *mR, double *out) {
  if (!prob_ok(P)) return ORC_EINVAL;
  long N = grid_N(P);
  int d = P->d, nc = P->n_c;
  double hd = cell_volume(P);
  double *mt = malloc(sizeof(double) * (long)(P->n_t + 1) * N);
  double *Rv = malloc(sizeof(double) * (long)nc * d * N);
  if (!mt || !Rv) { free(mt); free(Rv); return ORC_ENOMEM; }
  int st = orc_state(P, v, mT, mt, NULL);
  if (!st) st = orc_reg_apply(P, v, Rv);
  if (!st) {
    const double *m1 = mt + (long)P->n_t * N;
    double dist = 0.0, reg = 0.0;
    for (long x = 0; x < N; ++x) dist += (mR[x] - m1[x]) * (mR[x] - m1[x]);
    for (long q = 0; q < (long)nc * d * N; ++q) reg += v[q] * Rv[q];
    out[1] = 0.5 * hd * dist;
    out[2] = 0.5 * hd * reg;
    out[0] = out[1] + out[2];
  }
  free(mt);
  free(Rv);
  return st;
}

/* f_l = sum_j w_j b_l(t_j) lam_j grad m_j (trapezoid, reading R4), or the
 * discrete-adjoint form sum_j h/2 [b_l(t_j) lh_j grad m_j +
 * b_l(t_{j+1}) lam_{j+1} grad mh_{j+1}] when P->dto (test-only).
 * gm: (n_t+1) x d x N gradients of m_j; gmh: same for mh (dto only). */
static void body_force(const orc_prob *P, const double *ltraj, const double *lhat, const double *gm,
                       const double *gmh, double *f) {
  long N = grid_N(P);
  int d = P->d, nc = P->n_c, nt = P->n_t;
  double h = 1.0 / nt;
  memset(f, 0, sizeof(double) * (long)nc * d * N);
  double b[64], b2[64];
  if (!P->dto) {
    for (int j = 0; j <= nt; ++j) {
      double w = (j == 0 || j == nt) ? 0.5 * h : h;
      orc_cheb_eval(nc, j * h, b);
      const double *lj = ltraj + (long)j * N;
      const double *g = gm + (long)j * d * N;
#pragma omp parallel for schedule(static)
      for (long x = 0; x < N; ++x)
        for (int l = 0; l < nc; ++l)
          for (int i = 0; i < d; ++i) f[((long)l * d + i) * N + x] += w * b[l] * lj[x] * g[i * N + x];
    }
  } else {
    for (int j = 0; j < nt; ++j) {
      orc_cheb_eval(nc, j * h, b);
      orc_cheb_eval(nc, (j + 1) * h, b2);
      const double *lh = lhat + (long)j * N, *l1 = ltraj + (long)(j + 1) * N;
      const double *g0 = gm + (long)j * d * N, *g1 = gmh + (long)(j + 1) * d * N;
#pragma omp parallel for schedule(static)
      for (long x = 0; x < N; ++x)
        for (int l = 0; l < nc; ++l)
          for (int i = 0; i < d; ++i)
            f[((long)l * d + i) * N + x] +=
                0.5 * h * (b[l] * lh[x] * g0[i * N + x] + b2[l] * l1[x] * g1[i * N + x]);
    }
  }
}

/* out = beta sum C A v + K^gamma f (Eq. eliminated-control /
 * eliminated-icontrol with App. A Eq. control-equation-expansion) */
static int control_tail(const orc_prob *P, const double *v, double *f, double *out) {
  long N = grid_N(P);
  int d = P->d, nc = P->n_c;
  int st = orc_reg_apply(P, v, out);
  if (st) return st;
  double *kf = NULL;
  if (P->stokes) {
    kf = malloc(sizeof(double) * d * N);
    if (!kf) return ORC_ENOMEM;
  }
  for (int l = 0; l < nc && !st; ++l) {
    double *fl = f + (long)l * d * N;
    if (P->stokes) {
      st = orc_leray(P, fl, kf);
      fl = kf;
    }
    if (st) break;
    double *ol = out + (long)l * d * N;
#pragma omp parallel for schedule(static)
    for (long q = 0; q < d * N; ++q) ol[q] += fl[q];
  }
  free(kf);
  return st;
}

/* gradients of every stored state slot: gm[j] = grad m_j */
static int trajectory_gradients(const orc_prob *P, const double *mt, double *gm, int first) {
  long N = grid_N(P);
  int st = 0;
  for (int j = first; j <= P->n_t && !st; ++j)
    st = orc_grad(P, mt + (long)j * N, gm + (long)j * P->d * N);
  return st;
}

/* Reduced gradient g (Eq. first-order-control with Eq. eliminated-control and
 * App. A): state solve, lam_1 = m_R - m_1, adjoint solve, body force, tail.
 * J (may be NULL) receives the objective at v. */
int orc_gradient(const orc_prob *P, const double *v, const double *mT, const double *mR, double *g, double *J) {
  if (!prob_ok(P)) return ORC_EINVAL;
  long N = grid_N(P);
  int d = P->d, nc = P->n_c, nt = P->n_t;
  long T = nt + 1;
  double *mt = malloc(sizeof(double) * T * N), *lt = malloc(sizeof(double) * T * N);
  double *gm = malloc(sizeof(double) * T * d * N), *f = malloc(sizeof(double) * (long)nc * d * N);
  double *mh = NULL, *lh = NULL, *gmh = NULL;
  int st = (!mt || !lt || !gm || !f) ? ORC_ENOMEM : ORC_OK;
  if (!st && P->dto) {
    mh = malloc(sizeof(double) * T * N);
    lh = malloc(sizeof(double) * T * N);
    gmh = malloc(sizeof(double) * T * d * N);
    if (!mh || !lh || !gmh) st = ORC_ENOMEM;
  }
  if (!st) st = orc_state(P, v, mT, mt, mh);
  if (!st) {
    double *lend = lt + (long)nt * N;
    const double *m1 = mt + (long)nt * N;
    for (long x = 0; x < N; ++x) lend[x] = mR[x] - m1[x];
    double *tmp = malloc(sizeof(double) * N);
    if (!tmp) st = ORC_ENOMEM;
    else {
      memcpy(tmp, lend, sizeof(double) * N);
      st = orc_adjoint(P, v, tmp, lt, lh);
      free(tmp);
    }
  }
  if (!st) st = trajectory_gradients(P, mt, gm, 0);
  if (!st && P->dto) st = trajectory_gradients(P, mh, gmh, 1);
  if (!st) {
    body_force(P, lt, lh, gm, gmh, f);
    st = control_tail(P, v, f, g);
  }
  if (!st && J) {
    double hd = cell_volume(P);
    double *Rv = malloc(sizeof(double) * (long)nc * d * N);
    if (!Rv) st = ORC_ENOMEM;
    else {
      st = orc_reg_apply(P, v, Rv);
      const double *m1 = mt + (long)nt * N;
      double dist = 0.0, reg = 0.0;
      for (long x = 0; x < N; ++x) dist += (mR[x] - m1[x]) * (mR[x] - m1[x]);
      for (long q = 0; q < (long)nc * d * N; ++q) reg += v[q] * Rv[q];
      *J = 0.5 * hd * (dist + reg);
      free(Rv);
    }
  }
  free(mt); free(lt); free(gm); free(f); free(mh); free(lh); free(gmh);
  return st;
}

/* Gauss-Newton Hessian matvec (Alg. 2 with Eq. gauss-newton, all lambda
 * terms dropped; Sec. 3.2.2):
 *   incremental state  mt' = L(t) mt + s(t), s = -grad m . vt(t), mt_0 = 0,
 *   incremental adjoint backward from lt_1 = -mt_1 with D(t),
 *   out_l = beta sum C A vt_l' + K^gamma f~_l.
 * Heun for the incremental state: k1 = L_j mt_j + s_j,
 * k2 = L_{j+1}(mt_j + h k1) + s'_{j+1}, with s'_{j+1} = s_{j+1} (trapezoid
 * reading) or -grad mh_{j+1} . vt(t_{j+1}) (discrete adjoint, test-only). */
int orc_hessvec(const orc_prob *P, const double *v, const double *mT, const double *vt, double *out) {
  if (!prob_ok(P)) return ORC_EINVAL;
  long N = grid_N(P);
  int d = P->d, nc = P->n_c, nt = P->n_t;
  long T = nt + 1;
  double h = 1.0 / nt;
  double *mt = malloc(sizeof(double) * T * N), *gm = malloc(sizeof(double) * T * d * N);
  double *lt = malloc(sizeof(double) * T * N), *f = malloc(sizeof(double) * (long)nc * d * N);
  double *va = malloc(sizeof(double) * d * N), *vb = malloc(sizeof(double) * d * N);
  double *wa = malloc(sizeof(double) * d * N), *wb = malloc(sizeof(double) * d * N);
  double *y = malloc(sizeof(double) * N), *yh = malloc(sizeof(double) * N);
  double *k1 = malloc(sizeof(double) * N), *k2 = malloc(sizeof(double) * N);
  double *gt = malloc(sizeof(double) * d * N);
  double *mh = NULL, *gmh = NULL, *lh = NULL;
  int st = (!mt || !gm || !lt || !f || !va || !vb || !wa || !wb || !y || !yh || !k1 || !k2 || !gt) ? ORC_ENOMEM : 0;
  if (!st && P->dto) {
    mh = malloc(sizeof(double) * T * N);
    gmh = malloc(sizeof(double) * T * d * N);
    lh = malloc(sizeof(double) * T * N);
    if (!mh || !gmh || !lh) st = ORC_ENOMEM;
  }
  if (!st) st = orc_state(P, v, mT, mt, mh);
  if (!st) st = trajectory_gradients(P, mt, gm, 0);
  if (!st && P->dto) st = trajectory_gradients(P, mh, gmh, 1);
  /* incremental state, forward */
  if (!st) memset(y, 0, sizeof(double) * N);
  for (int j = 0; j < nt && !st; ++j) {
    velocity_at(P, v, j * h, va);
    velocity_at(P, v, (j + 1) * h, vb);
    velocity_at(P, vt, j * h, wa);
    velocity_at(P, vt, (j + 1) * h, wb);
    const double *g0 = gm + (long)j * d * N;
    const double *g1 = P->dto ? gmh + (long)(j + 1) * d * N : gm + (long)(j + 1) * d * N;
    st = apply_L(P, va, y, k1, gt);
    if (st) break;
#pragma omp parallel for schedule(static)
    for (long x = 0; x < N; ++x) {
      double s = 0.0;
      for (int i = 0; i < d; ++i) s += g0[i * N + x] * wa[i * N + x];
      k1[x] -= s;
      yh[x] = y[x] + h * k1[x];
    }
    st = apply_L(P, vb, yh, k2, gt);
    if (st) break;
#pragma omp parallel for schedule(static)
    for (long x = 0; x < N; ++x) {
      double s = 0.0;
      for (int i = 0; i < d; ++i) s += g1[i * N + x] * wb[i * N + x];
      k2[x] -= s;
      y[x] = y[x] + 0.5 * h * (k1[x] + k2[x]);
    }
  }
  /* incremental adjoint, backward from -mt_1 */
  if (!st) {
#pragma omp parallel for schedule(static)
    for (long x = 0; x < N; ++x) y[x] = -y[x];
    st = orc_adjoint(P, v, y, lt, lh);
  }
  if (!st) {
    body_force(P, lt, lh, gm, gmh, f);
    st = control_tail(P, vt, f, out);
  }
  free(mt); free(gm); free(lt); free(f); free(va); free(vb); free(wa); free(wb);
  free(y); free(yh); free(k1); free(k2); free(gt); free(mh); free(gmh); free(lh);
  return st;
}

/* Full Newton Hessian matvec (Eq. sec-order-opt-cond with the pressure
 * eliminated, Eq. eliminated-icontrol; trapezoid quadrature only):
 *   incremental state   as in orc_hessvec,
 *   incremental adjoint -d/dt lt - div(v lt) - div(vt lam) = 0, lt_1 = -mt_1,
 *                       Heun backward with the source s(t_j) = div(vt(t_j) lam_j),
 *   body force          f~_l = sum_j w_j b_l(t_j) [lt_j grad m_j + lam_j grad mt_j],
 *   out_l = beta sum C A vt_l' + K^gamma f~_l,
 * with lam the adjoint of orc_gradient (lam_1 = m_R - m_1). */
int orc_hessvec_newton(const orc_prob *P, const double *v, const double *mT, const double *mR, const double *vt,
                       double *out) {
  if (!prob_ok(P) || P->dto) return ORC_EINVAL;
  long N = grid_N(P);
  int d = P->d, nc = P->n_c, nt = P->n_t;
  long T = nt + 1;
  double h = 1.0 / nt;
  double *mt = malloc(sizeof(double) * T * N), *gm = malloc(sizeof(double) * T * d * N);
  double *lam = malloc(sizeof(double) * T * N), *mtil = malloc(sizeof(double) * T * N);
  double *ltil = malloc(sizeof(double) * T * N), *f = calloc((long)nc * d * N, sizeof(double));
  double *va = malloc(sizeof(double) * d * N), *vb = malloc(sizeof(double) * d * N);
  double *wa = malloc(sizeof(double) * d * N), *wb = malloc(sizeof(double) * d * N);
  double *k1 = malloc(sizeof(double) * N), *k2 = malloc(sizeof(double) * N), *yh = malloc(sizeof(double) * N);
  double *sa = malloc(sizeof(double) * N), *sb = malloc(sizeof(double) * N);
  double *gt = malloc(sizeof(double) * d * N), *wtmp = malloc(sizeof(double) * d * N);
  int st = (!mt || !gm || !lam || !mtil || !ltil || !f || !va || !vb || !wa || !wb || !k1 || !k2 || !yh || !sa || !sb ||
            !gt || !wtmp) ? ORC_ENOMEM : 0;
  /* state, its gradients, and the adjoint from lam_1 = m_R - m_1 */
  if (!st) st = orc_state(P, v, mT, mt, NULL);
  if (!st) st = trajectory_gradients(P, mt, gm, 0);
  if (!st) {
    double *tmp = malloc(sizeof(double) * N);
    if (!tmp) st = ORC_ENOMEM;
    else {
      for (long x = 0; x < N; ++x) tmp[x] = mR[x] - mt[(long)nt * N + x];
      st = orc_adjoint(P, v, tmp, lam, NULL);
      free(tmp);
    }
  }
  /* incremental state, forward (as in orc_hessvec), keeping every node */
  if (!st) memset(mtil, 0, sizeof(double) * N);
  for (int j = 0; j < nt && !st; ++j) {
    const double *y = mtil + (long)j * N;
    double *yn = mtil + (long)(j + 1) * N;
    velocity_at(P, v, j * h, va);
    velocity_at(P, v, (j + 1) * h, vb);
    velocity_at(P, vt, j * h, wa);
    velocity_at(P, vt, (j + 1) * h, wb);
    const double *g0 = gm + (long)j * d * N, *g1 = gm + (long)(j + 1) * d * N;
    st = apply_L(P, va, y, k1, gt);
    if (st) break;
    for (long x = 0; x < N; ++x) {
      double s = 0.0;
      for (int i = 0; i < d; ++i) s += g0[i * N + x] * wa[i * N + x];
      k1[x] -= s;
      yh[x] = y[x] + h * k1[x];
    }
    st = apply_L(P, vb, yh, k2, gt);
    if (st) break;
    for (long x = 0; x < N; ++x) {
      double s = 0.0;
      for (int i = 0; i < d; ++i) s += g1[i * N + x] * wb[i * N + x];
      k2[x] -= s;
      yn[x] = y[x] + 0.5 * h * (k1[x] + k2[x]);
    }
  }
  /* incremental adjoint, backward from -mt_1, with the source div(vt lam) */
  if (!st) {
    for (long x = 0; x < N; ++x) ltil[(long)nt * N + x] = -mtil[(long)nt * N + x];
    velocity_at(P, vt, 1.0, wb);
    st = apply_D(P, wb, lam + (long)nt * N, sb, wtmp);
  }
  for (int j = nt - 1; j >= 0 && !st; --j) {
    const double *l1 = ltil + (long)(j + 1) * N;
    double *l0 = ltil + (long)j * N;
    velocity_at(P, v, (j + 1) * h, vb);
    velocity_at(P, v, j * h, va);
    velocity_at(P, vt, j * h, wa);
    st = apply_D(P, wa, lam + (long)j * N, sa, wtmp); /* source at t_j */
    if (st) break;
    st = apply_D(P, vb, l1, k1, wtmp);
    if (st) break;
    for (long x = 0; x < N; ++x) {
      k1[x] += sb[x];
      yh[x] = l1[x] + h * k1[x];
    }
    st = apply_D(P, va, yh, k2, wtmp);
    if (st) break;
    for (long x = 0; x < N; ++x) {
      k2[x] += sa[x];
      l0[x] = l1[x] + 0.5 * h * (k1[x] + k2[x]);
    }
    double *t = sa;
    sa = sb;
    sb = t; /* the source at t_j is the next step's source at t_{j+1} */
  }
  /* body force f~_l = sum_j w_j b_l(t_j) [lt_j grad m_j + lam_j grad mt_j] */
  double b[64];
  for (int j = 0; j <= nt && !st; ++j) {
    double w = (j == 0 || j == nt) ? 0.5 * h : h;
    orc_cheb_eval(nc, j * h, b);
    st = orc_grad(P, mtil + (long)j * N, gt);
    if (st) break;
    const double *lt = ltil + (long)j * N, *lj = lam + (long)j * N, *g = gm + (long)j * d * N;
    for (long x = 0; x < N; ++x)
      for (int l = 0; l < nc; ++l)
        for (int i = 0; i < d; ++i)
          f[((long)l * d + i) * N + x] += w * b[l] * (lt[x] * g[i * N + x] + lj[x] * gt[i * N + x]);
  }
  if (!st) st = control_tail(P, vt, f, out);
  free(mt); free(gm); free(lam); free(mtil); free(ltil); free(f); free(va); free(vb); free(wa); free(wb);
  free(k1); free(k2); free(yh); free(sa); free(sb); free(gt); free(wtmp);
  return st;
}

/* ------------------------------------------------------------------ */
/* Deformation gradient (App. D Eq. def-grad) and CFL number (Sec. 3.3.1) */
/* ------------------------------------------------------------------ */

/* dF/dt = -(v . grad) F + (grad v) F, F_0 = I, Heun in time;
 * (grad v)_{ik} = d v_i / d x_k. detF: N values of det F_1. */
static int defgrad(const orc_prob *P, const double *v, double *Fout, double *detF) {
  if (!prob_ok(P)) return ORC_EINVAL;
  long N = grid_N(P);
  int d = P->d, nt = P->n_t, nc = P->n_c, dd = d * d;
  double h = 1.0 / nt;
  /* gradients of every coefficient field: gv[l][i][k] = d_k v_{l,i} */
  double *gv = malloc(sizeof(double) * (long)nc * dd * N);
  double *F = malloc(sizeof(double) * dd * N), *Fh = malloc(sizeof(double) * dd * N);
  double *K1 = malloc(sizeof(double) * dd * N), *K2 = malloc(sizeof(double) * dd * N);
  double *vt = malloc(sizeof(double) * d * N), *gt = malloc(sizeof(double) * d * N);
  double *Gt = malloc(sizeof(double) * dd * N), *k = malloc(sizeof(double) * N);
  int st = (!gv || !F || !Fh || !K1 || !K2 || !vt || !gt || !Gt || !k) ? ORC_ENOMEM : 0;
  for (int l = 0; l < nc && !st; ++l)
    for (int i = 0; i < d && !st; ++i)
      st = orc_grad(P, v + ((long)l * d + i) * N, gv + ((long)l * dd + i * d) * N);
  if (!st) {
#pragma omp parallel for schedule(static)
    for (long x = 0; x < N; ++x)
      for (int a = 0; a < d; ++a)
        for (int c = 0; c < d; ++c) F[(a * d + c) * N + x] = (a == c) ? 1.0 : 0.0;
  }
  double b[64];
  for (int j = 0; j < nt && !st; ++j) {
    for (int stage = 0; stage < 2 && !st; ++stage) {
      double t = (j + stage) * h;
      const double *Fin = stage == 0 ? F : Fh;
      double *Kout = stage == 0 ? K1 : K2;
      velocity_at(P, v, t, vt);
      orc_cheb_eval(nc, t, b);
#pragma omp parallel for schedule(static)
      for (long x = 0; x < N; ++x)
        for (int q = 0; q < dd; ++q) {
          double s = 0.0;
          for (int l = 0; l < nc; ++l) s += b[l] * gv[((long)l * dd + q) * N + x];
          Gt[q * N + x] = s;
        }
      for (int q = 0; q < dd && !st; ++q) {
        st = apply_L(P, vt, Fin + q * N, k, gt);
        if (st) break;
        int a = q / d, c = q % d;
#pragma omp parallel for schedule(static)
        for (long x = 0; x < N; ++x) {
          double s = k[x];
          for (int m = 0; m < d; ++m) s += Gt[(a * d + m) * N + x] * Fin[(m * d + c) * N + x];
          Kout[q * N + x] = s;
        }
      }
      if (st) break;
      if (stage == 0) {
#pragma omp parallel for schedule(static)
        for (long q = 0; q < dd * N; ++q) Fh[q] = F[q] + h * K1[q];
      } else {
#pragma omp parallel for schedule(static)
        for (long q = 0; q < dd * N; ++q) F[q] = F[q] + 0.5 * h * (K1[q] + K2[q]);
      }
    }
  }
  if (!st && Fout) memcpy(Fout, F, sizeof(double) * dd * N);
  if (!st && detF) {
#pragma omp parallel for schedule(static)
    for (long x = 0; x < N; ++x) {
      if (d == 2) {
        detF[x] = F[0 * N + x] * F[3 * N + x] - F[1 * N + x] * F[2 * N + x];
      } else {
        double a00 = F[0 * N + x], a01 = F[1 * N + x], a02 = F[2 * N + x];
        double a10 = F[3 * N + x], a11 = F[4 * N + x], a12 = F[5 * N + x];
        double a20 = F[6 * N + x], a21 = F[7 * N + x], a22 = F[8 * N + x];
        detF[x] = a00 * (a11 * a22 - a12 * a21) - a01 * (a10 * a22 - a12 * a20) + a02 * (a10 * a21 - a11 * a20);
      }
    }
  }
  free(gv); free(F); free(Fh); free(K1); free(K2); free(vt); free(gt); free(Gt); free(k);
  return st;
}

int orc_detF(const orc_prob *P, const double *v, double *detF) { return defgrad(P, v, NULL, detF); }

/* F_1 itself: d*d fields, F[(a*d + c)*N + x] = F_ac */
int orc_defgrad(const orc_prob *P, const double *v, double *F) { return defgrad(P, v, F, NULL); }

/* Grid-angle measure of the deformation (Sec. 3.3.5 "Regularization", the
 * acute angle of a deformed grid element): the edges e_c of a cell map to the
 * columns F_1 e_c; per point, the smallest over column pairs of
 * min(theta, pi - theta), theta the angle between the two columns. angle: N
 * values in [0, pi/2]; pi/2 for F = I. */
int orc_grid_angle(const orc_prob *P, const double *v, double *angle) {
  if (!prob_ok(P)) return ORC_EINVAL;
  long N = grid_N(P);
  int d = P->d;
  double *F = malloc(sizeof(double) * d * d * N);
  if (!F) return ORC_ENOMEM;
  int st = defgrad(P, v, F, NULL);
  if (!st) {
#pragma omp parallel for schedule(static)
    for (long x = 0; x < N; ++x) {
      double best = 0.5 * M_PI;
      for (int c1 = 0; c1 < d; ++c1)
        for (int c2 = c1 + 1; c2 < d; ++c2) {
          double dot12 = 0.0, n1 = 0.0, n2 = 0.0;
          for (int a = 0; a < d; ++a) {
            double f1 = F[(a * d + c1) * N + x], f2 = F[(a * d + c2) * N + x];
            dot12 += f1 * f2;
            n1 += f1 * f1;
            n2 += f2 * f2;
          }
          double cs = dot12 / sqrt(n1 * n2);
          if (cs > 1.0) cs = 1.0;
          if (cs < -1.0) cs = -1.0;
          double th = acos(cs);
          double acute = th < 0.5 * M_PI ? th : M_PI - th;
          if (acute < best) best = acute;
        }
      angle[x] = best;
    }
  }
  free(F);
  return st;
}

/* Deformation map (App. D Eq. displacement): du/dt + (grad u) v = v, u_0 = 0,
 * componentwise du_i/dt = -v . grad u_i + v_i, Heun steps on the time nodes
 * as the state equation. u: d fields, the displacement u_1 (y = x - u_1). */
int orc_displacement(const orc_prob *P, const double *v, double *u) {
  if (!prob_ok(P)) return ORC_EINVAL;
  long N = grid_N(P);
  int d = P->d, nt = P->n_t;
  double h = 1.0 / nt;
  double *va = malloc(sizeof(double) * d * N), *vb = malloc(sizeof(double) * d * N);
  double *k1 = malloc(sizeof(double) * N), *k2 = malloc(sizeof(double) * N), *yh = malloc(sizeof(double) * N);
  double *gt = malloc(sizeof(double) * d * N);
  int st = (!va || !vb || !k1 || !k2 || !yh || !gt) ? ORC_ENOMEM : 0;
  if (!st) memset(u, 0, sizeof(double) * d * N);
  for (int j = 0; j < nt && !st; ++j) {
    velocity_at(P, v, j * h, va);
    velocity_at(P, v, (j + 1) * h, vb);
    for (int i = 0; i < d && !st; ++i) {
      double *ui = u + (long)i * N;
      st = apply_L(P, va, ui, k1, gt);
      if (st) break;
      for (long x = 0; x < N; ++x) {
        k1[x] += va[i * N + x];
        yh[x] = ui[x] + h * k1[x];
      }
      st = apply_L(P, vb, yh, k2, gt);
      if (st) break;
      for (long x = 0; x < N; ++x) {
        k2[x] += vb[i * N + x];
        ui[x] = ui[x] + 0.5 * h * (k1[x] + k2[x]);
      }
    }
  }
  free(va); free(vb); free(k1); free(k2); free(yh); free(gt);
  return st;
}

/* Gaussian presmoothing (Sec. 3.3.5 "Presmoothing"): out = G_sigma * in on the
 * periodic domain, i.e. the Fourier multiplier exp(-sigma^2 |k|^2 / 2) with the
 * full wavenumbers (Nyquist modes included). */
int orc_smooth(const orc_prob *P, double sigma, const double *in, double *out) {
  if (!prob_ok(P) || !(sigma >= 0.0)) return ORC_EINVAL;
  long N = grid_N(P);
  double *U = malloc(sizeof(double) * 2 * N);
  if (!U) return ORC_ENOMEM;
  int st = to_spectrum(P, in, U);
  if (!st) {
#pragma omp parallel for schedule(static)
    for (long x = 0; x < N; ++x) {
      int j[3];
      unflatten(P, x, j);
      double kk = 0.0;
      for (int i = 0; i < P->d; ++i) {
        double k = wavenumber(j[i], P->n[i]);
        kk += k * k;
      }
      double g = exp(-0.5 * sigma * sigma * kk);
      U[2 * x] *= g;
      U[2 * x + 1] *= g;
    }
    st = from_spectrum(P, U, out);
  }
  free(U);
  return st;
}

/* CFL number h_t * max_j max_i ||v_i(t_j)||_inf / h_x^i over the time nodes */
double orc_cfl(const orc_prob *P, const double *v) {
  long N = grid_N(P);
  int d = P->d;
  double *vt = malloc(sizeof(double) * d * N);
  if (!vt) return -1.0;
  double c = 0.0, h = 1.0 / P->n_t;
  for (int j = 0; j <= P->n_t; ++j) {
    velocity_at(P, v, j * h, vt);
    for (int i = 0; i < d; ++i) {
      double hx = 2.0 * M_PI / P->n[i], mx = 0.0;
      for (long x = 0; x < N; ++x) mx = fmax(mx, fabs(vt[i * N + x]));
      c = fmax(c, h * mx / hx);
    }
  }
  free(vt);
  return c;
}

/* ------------------------------------------------------------------ */
/* Inexact Gauss-Newton-Krylov solve (Alg. 1; PCG per Eq.              */
/* termination-criterion-ksm; Armijo backtracking, Sec. 3.2); with     */
/* opts.newton the full Newton matvec (N-PCG of Sec. 4)                */
/* ------------------------------------------------------------------ */

static double dot(long n, const double *a, const double *b) {
  double s = 0.0;
  for (long q = 0; q < n; ++q) s += a[q] * b[q];
  return s;
}

static double norm_inf(long n, const double *a) {
  double s = 0.0;
  for (long q = 0; q < n; ++q) s = fmax(s, fabs(a[q]));
  return s;
}

/* Termination test at iterate k (Eq. stopping-criteria / Eq. converged, or
 * the relative gradient reduction of Sec. 3.3.5). Returns 1 to stop; *flags
 * gets the criteria that hold; *maxed is set when only the iteration cap
 * stops the solve. */
static int stop_test(const orc_opts *O, const orc_report *R, int k, double ginf, int *flags, int *maxed) {
  *flags = 0;
  *maxed = 0;
  if (O->stop_rule == 0) {
    if (ginf <= O->grad_rtol * R->g0_inf) return 1;
    if (k >= O->max_outer) {
      *maxed = 1;
      return 1;
    }
    return 0;
  }
  double tau = O->tau_J, one_J0 = 1.0 + R->J0;
  if (k >= 1 && R->J_prev - R->J < tau * one_J0) *flags |= 1;          /* C1 */
  if (k >= 1 && R->dv_inf < sqrt(tau) * (1.0 + R->v_inf)) *flags |= 2; /* C2 */
  if (ginf < cbrt(tau) * one_J0) *flags |= 4;                          /* C3 */
  if (ginf < 1e3 * DBL_EPSILON) *flags |= 8;                           /* C4 */
  if (k > O->max_outer) *flags |= 16;                                  /* C5 */
  int conv = ((*flags & 7) == 7) || (*flags & 8);
  if (conv) return 1;
  if (*flags & 16) {
    *maxed = 1;
    return 1;
  }
  return 0;
}

/* Outer loop (Alg. 1): the search direction is the inexact (G)N step from
 * PCG on H s = -g (Nocedal & Wright Alg. 5.3) or, with opts.picard, the
 * Picard update s = -P^{-1} g (Eq. picard; App. C: the difference between the
 * Picard iterate -(beta C (x) A)^{-1} K f and v_k), scaled by the step memory
 * alpha~; then CFL halving and Armijo backtracking from alpha = 1. */
int orc_solve(const orc_prob *P, const orc_opts *O, const double *mT, const double *mR, double *v, orc_report *R) {
  if (!prob_ok(P)) return ORC_EINVAL;
  if (O->newton && P->dto) return ORC_EINVAL;
  long N = grid_N(P);
  long n = (long)P->n_c * P->d * N;
  double hd = cell_volume(P);
  double *g = malloc(sizeof(double) * n), *s = malloc(sizeof(double) * n);
  double *r = malloc(sizeof(double) * n), *z = malloc(sizeof(double) * n);
  double *p = malloc(sizeof(double) * n), *Hp = malloc(sizeof(double) * n);
  double *vtrial = malloc(sizeof(double) * n);
  memset(R, 0, sizeof(*R));
  int st = (!g || !s || !r || !z || !p || !Hp || !vtrial) ? ORC_ENOMEM : 0;
  double J = 0.0, out3[3];
  long maxit = O->pcg_maxit > 0 ? O->pcg_maxit : n;
  double amem = 1.0;
  R->alpha_mem = amem;
  if (!st) st = orc_gradient(P, v, mT, mR, g, &J);
  R->n_pde += 2;
  if (!st) {
    R->J0 = J;
    R->g0_inf = norm_inf(n, g);
    R->g0_2 = sqrt(dot(n, g, g));
    R->v_inf = norm_inf(n, v);
  }
  int k = 0, maxed = 0;
  while (!st) {
    double ginf = norm_inf(n, g), g2 = sqrt(dot(n, g, g));
    R->g_inf = ginf;
    R->g_2 = g2;
    R->J = J;
    if (stop_test(O, R, k, ginf, &R->stop_flags, &maxed)) break;
    if (O->picard) {
      st = orc_precond(P, g, s);
      if (st) break;
      double sc = O->step_memory ? -amem : -1.0;
      for (long q = 0; q < n; ++q) s[q] *= sc;
    } else {
      /* PCG on H s = -g from s = 0 */
      double eta = fmin(0.5, sqrt(g2 / R->g0_2));
      memset(s, 0, sizeof(double) * n);
      memcpy(r, g, sizeof(double) * n); /* r_0 = H s_0 + g = g */
      st = orc_precond(P, r, z);
      for (long q = 0; q < n && !st; ++q) p[q] = -z[q];
      double rz = dot(n, r, z);
      for (long it = 0; it < maxit && !st; ++it) {
        if (sqrt(dot(n, r, r)) <= eta * g2) break;
        st = O->newton ? orc_hessvec_newton(P, v, mT, mR, p, Hp) : orc_hessvec(P, v, mT, p, Hp);
        R->matvecs += 1;
        R->n_pde += 2;
        R->pcg_iters += 1;
        if (st) break;
        double pHp = dot(n, p, Hp);
        if (pHp <= 0.0) {
          if (it == 0) memcpy(s, p, sizeof(double) * n);
          break;
        }
        double alpha = rz / pHp;
        for (long q = 0; q < n; ++q) {
          s[q] += alpha * p[q];
          r[q] += alpha * Hp[q];
        }
        st = orc_precond(P, r, z);
        if (st) break;
        double rz_new = dot(n, r, z);
        double bta = rz_new / rz;
        rz = rz_new;
        for (long q = 0; q < n; ++q) p[q] = -z[q] + bta * p[q];
      }
      if (st) break;
    }
    /* keep v + s inside the CFL bound by halving s (Sec. 3.3.5) */
    if (O->cfl_max > 0.0) {
      for (int halvings = 0;; ++halvings) {
        for (long q = 0; q < n; ++q) vtrial[q] = v[q] + s[q];
        if (orc_cfl(P, vtrial) <= O->cfl_max) break;
        if (halvings == 30) { /* 30 halvings of this step did not suffice */
          st = ORC_ECFL;
          break;
        }
        for (long q = 0; q < n; ++q) s[q] *= 0.5;
        R->cfl_halvings += 1;
      }
      if (st) break;
    }
    /* Armijo backtracking from alpha = 1 */
    double slope = hd * dot(n, g, s);
    double alpha = 1.0, Jt = 0.0;
    int accepted = 0;
    for (int t = 0; t < O->max_backtracks; ++t) {
      for (long q = 0; q < n; ++q) vtrial[q] = v[q] + alpha * s[q];
      st = orc_objective(P, vtrial, mT, mR, out3);
      R->ls_trials += 1;
      R->n_pde += 1;
      if (st) break;
      Jt = out3[0];
      if (Jt <= J + O->armijo_c1 * alpha * slope) {
        accepted = 1;
        break;
      }
      alpha *= O->backtrack;
    }
    if (st) break;
    if (!accepted) {
      st = ORC_ELINESEARCH;
      break;
    }
    /* step memory: double after a full step, else scale by the accepted alpha */
    if (O->picard && O->step_memory) amem = (alpha == 1.0) ? 2.0 * amem : amem * alpha;
    R->alpha_mem = amem;
    double dv = 0.0;
    for (long q = 0; q < n; ++q) dv = fmax(dv, fabs(vtrial[q] - v[q]));
    memcpy(v, vtrial, sizeof(double) * n);
    R->dv_inf = dv;
    R->v_inf = norm_inf(n, v);
    R->J_prev = J;
    st = orc_gradient(P, v, mT, mR, g, &J);
    R->n_pde += 2;
    k += 1;
  }
  R->outer = k;
  if (!st && maxed) st = ORC_EMAXIT;
  R->status = st;
  free(g); free(s); free(r); free(z); free(p); free(Hp); free(vtrial);
  return st;
}

/* Lanczos tridiagonalisation (Sec. 3.3.5 "Regularization": the condition
 * number of the Hessian estimated with the Lanczos algorithm, Golub & Van
 * Loan Sec. 9.1): k steps of the three-term recurrence on the Hessian at v
 * (Gauss-Newton, or full Newton with mR when newton = 1), from q0. With
 * precond = 1 the recurrence runs on P^{-1} H in the P inner product
 * (P^{-1} = orc_precond). Plain coefficient-vector inner products, no
 * reorthogonalisation. alpha[j] = q_j^T H q_j, beta[j] couples q_j and
 * q_{j+1}; *steps = steps completed (fewer than k after a breakdown
 * beta = 0). The eigenvalues of the tridiagonal matrix are the Ritz values. */
int orc_lanczos(const orc_prob *P, const double *v, const double *mT, const double *mR, int newton,
                const double *q0, int k, int precond, double *alpha, double *beta, int *steps) {
  if (!prob_ok(P) || k < 1 || (newton && (P->dto || !mR))) return ORC_EINVAL;
  long n = (long)P->n_c * P->d * grid_N(P);
  double *q = malloc(sizeof(double) * n), *u = malloc(sizeof(double) * n);
  double *up = calloc(n, sizeof(double));
  double *w = malloc(sizeof(double) * n), *z = malloc(sizeof(double) * n);
  int st = (!q || !u || !up || !w || !z) ? ORC_ENOMEM : 0;
  *steps = 0;
  /* q_0 (primal) and u_0 = P q_0 (dual); without precond u = q */
  if (!st) {
    memcpy(u, q0, sizeof(double) * n);
    if (precond) st = orc_precond(P, u, q);
    else memcpy(q, u, sizeof(double) * n);
  }
  if (!st) {
    double nrm = sqrt(dot(n, u, q));
    if (!(nrm > 0.0)) st = ORC_EINVAL;
    for (long i = 0; i < n && !st; ++i) {
      q[i] /= nrm;
      u[i] /= nrm;
    }
  }
  double bprev = 0.0;
  for (int j = 0; j < k && !st; ++j) {
    st = newton ? orc_hessvec_newton(P, v, mT, mR, q, w) : orc_hessvec(P, v, mT, q, w);
    if (st) break;
    for (long i = 0; i < n; ++i) w[i] -= bprev * up[i];
    double a = dot(n, q, w);
    for (long i = 0; i < n; ++i) w[i] -= a * u[i];
    if (precond) st = orc_precond(P, w, z);
    else memcpy(z, w, sizeof(double) * n);
    if (st) break;
    double b2 = dot(n, w, z);
    double b = b2 > 0.0 ? sqrt(b2) : 0.0;
    alpha[j] = a;
    beta[j] = b;
    *steps = j + 1;
    if (b == 0.0) break;
    for (long i = 0; i < n; ++i) {
      up[i] = u[i];
      u[i] = w[i] / b;
      q[i] = z[i] / b;
    }
    bprev = b;
  }
  free(q); free(u); free(up); free(w); free(z);
  return st;
}

/* Parameter continuation in beta (Sec. 3.3.5 "Regularization"): solve at
 * beta0, divide beta by 10 while min det F_1 >= eps_F (and the smallest grid
 * angle >= eps_theta when eps_theta > 0), then bisect between the last
 * accepted and the breaching beta until beta would change by less than
 * beta_rtol times the first breaching beta. The reduction also ends at
 * beta_min or when the relative L2 distance ||m_R - m_1|| / ||m_R - m_T||
 * drops by less than the fraction dist_rtol. Each solve starts from the last
 * accepted solution (from v before any); with cfl_target > 0 a solution above
 * it raises n_t to ceil(n_t CFL / cfl_target) (at least n_t + 1) and solves
 * again at the same beta. On return v is the accepted solution. */
typedef struct {
  double beta0, beta_min, eps_F, eps_theta, beta_rtol, dist_rtol, cfl_target;
  int max_solves;
} orc_cont_opts;

typedef struct {
  int found, stop, solves, n_t;
  double beta, beta_breach, detF_min, angle_min, dist;
  int n_trace;
  double trace_beta[64], trace_detF[64], trace_angle[64], trace_dist[64];
  int trace_ok[64];
} orc_cont_report;

int orc_continuation(const orc_prob *P0, const orc_opts *O, const orc_cont_opts *C, const double *mT,
                     const double *mR, double *v, orc_cont_report *R) {
  if (!prob_ok(P0)) return ORC_EINVAL;
  orc_prob P = *P0;
  long N = grid_N(&P);
  long n = (long)P.n_c * P.d * N;
  double *vstart = malloc(sizeof(double) * n), *vgood = malloc(sizeof(double) * n);
  double *det = malloc(sizeof(double) * N), *ang = malloc(sizeof(double) * N);
  int st = (!vstart || !vgood || !det || !ang) ? ORC_ENOMEM : 0;
  memset(R, 0, sizeof(*R));
  double base = 0.0;
  for (long x = 0; x < N; ++x) base += (mR[x] - mT[x]) * (mR[x] - mT[x]);
  if (!st) memcpy(vstart, v, sizeof(double) * n);
  int have_good = 0, bisect = 0;
  double beta_good = 0.0, beta_bad = 0.0, dist_prev = -1.0, beta = C->beta0;
  while (!st) {
    if (R->solves >= C->max_solves) {
      R->stop = 4;
      break;
    }
    P.beta = beta;
    memcpy(v, have_good ? vgood : vstart, sizeof(double) * n);
    orc_report sr;
    int ss = orc_solve(&P, O, mT, mR, v, &sr);
    R->solves += 1;
    /* a solve ended by the iteration cap or a failed line search keeps its last iterate */
    if (ss != 0 && ss != ORC_EMAXIT && ss != ORC_ELINESEARCH) {
      st = ss;
      break;
    }
    if (C->cfl_target > 0.0) {
      double cf = orc_cfl(&P, v);
      if (cf > C->cfl_target) {
        int want = (int)ceil(P.n_t * cf / C->cfl_target);
        P.n_t = want > P.n_t + 1 ? want : P.n_t + 1;
        continue;
      }
    }
    double out3[3];
    st = orc_objective(&P, v, mT, mR, out3);
    if (!st) st = orc_detF(&P, v, det);
    if (!st) st = orc_grid_angle(&P, v, ang);
    if (st) break;
    double dmin = det[0], amin = ang[0];
    for (long x = 1; x < N; ++x) {
      dmin = fmin(dmin, det[x]);
      amin = fmin(amin, ang[x]);
    }
    double dist = base > 0.0 ? sqrt((2.0 * out3[1] / cell_volume(&P)) / base) : 0.0;
    int ok = dmin >= C->eps_F && (C->eps_theta <= 0.0 || amin >= C->eps_theta);
    if (R->n_trace < 64) {
      int t = R->n_trace++;
      R->trace_beta[t] = beta;
      R->trace_detF[t] = dmin;
      R->trace_angle[t] = amin;
      R->trace_dist[t] = dist;
      R->trace_ok[t] = ok;
    }
    if (ok) {
      have_good = 1;
      beta_good = beta;
      memcpy(vgood, v, sizeof(double) * n);
      R->detF_min = dmin;
      R->angle_min = amin;
      R->dist = dist;
    }
    if (!bisect) {
      if (ok) {
        if (dist_prev > 0.0 && dist_prev - dist < C->dist_rtol * dist_prev) {
          R->stop = 2;
          break;
        }
        dist_prev = dist;
        if (beta / 10.0 < C->beta_min) {
          R->stop = 1;
          break;
        }
        beta /= 10.0;
        continue;
      }
      R->beta_breach = beta;
      if (!have_good) {
        R->stop = 3;
        break;
      }
      beta_bad = beta;
      bisect = 1;
    } else if (ok) {
      beta_good = beta;
    } else {
      beta_bad = beta;
    }
    double next = 0.5 * (beta_good + beta_bad);
    if (fabs(next - beta) < C->beta_rtol * R->beta_breach) {
      R->stop = 0;
      break;
    }
    beta = next;
  }
  if (!st) {
    R->found = have_good;
    if (have_good) memcpy(v, vgood, sizeof(double) * n);
    R->beta = have_good ? beta_good : beta;
    R->n_t = P.n_t;
  }
  free(vstart); free(vgood); free(det); free(ang);
  return st;
}

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
