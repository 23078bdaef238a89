// pointwise.cu -- pointwise stages of the transport solves and the vector
// kernels of the Krylov/Newton loops (Mang & Biros, Sec. 3.2-3.3).
//
// Heun's RK2 (reading of "explicit second-order Runge-Kutta", Sec. 3.3.1):
//   k1 = F(t_j, y_j), yh = y_j + h k1, k2 = F(t_{j+1}, yh),
//   y_{j+1} = y_j + h/2 (k1 + k2) = acc + h/2 k2 with acc = y_j + h/2 k1.
// The stage kernels below take the spectral derivatives of the current stage
// input and form the right-hand sides of
//   state        m'  = -v . grad m                      (Eq. first-order-forward)
//   incr. state  m~' = -v . grad m~ - grad m . v~        (Eq. gauss-newton)
// together with the Runge-Kutta combination.
#include <float.h>

#include "pointwise.h"

namespace reg {

namespace {

inline unsigned nblk(long n, int bs = 256) {
  long b = (n + bs - 1) / bs;
  return (unsigned)(b < 1 ? 1 : b);
}

template <typename T, typename S>
__global__ void k_vel_at(const S* __restrict__ coef, int nc, Coefs b, T* __restrict__ out, long dN) {
  long x = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= dN) return;
  double s = 0.0;
  for (int l = 0; l < nc; ++l) s += b.c[l] * (double)coef[l * dN + x];
  out[x] = (T)s;
}

template <typename S, typename T>
__global__ void k_convert(const S* __restrict__ in, T* __restrict__ out, long n) {
  long x = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (x < n) out[x] = (T)in[x];
}

// k = -sum_i v_i G_i - [sum_i gm_i w_i]; Heun stage 1 or 2 update.
template <typename T, bool SRC, bool STAGE1>
__global__ void k_stage(const T* __restrict__ G, const T* __restrict__ vt, const T* __restrict__ gm,
                        const T* __restrict__ wt, const T* __restrict__ y, T h, T* __restrict__ yh,
                        T* __restrict__ acc, int d, long N) {
  long x = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= N) return;
  T k = 0;
  if (G)
    for (int i = 0; i < d; ++i) k -= vt[i * N + x] * G[i * N + x];
  if (SRC)
    for (int i = 0; i < d; ++i) k -= gm[i * N + x] * wt[i * N + x];
  if (STAGE1) {
    T yv = y ? y[x] : (T)0;
    yh[x] = yv + h * k;
    acc[x] = yv + (T)0.5 * h * k;
  } else {
    yh[x] = y[x] + (T)0.5 * h * k;  // y holds acc here; yh is the new state
  }
}

template <typename T>
__global__ void k_dot_fields(const T* __restrict__ a, const T* __restrict__ b, T* __restrict__ out, int d, long N) {
  long x = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= N) return;
  T s = 0;
  for (int i = 0; i < d; ++i) s += a[i * N + x] * b[i * N + x];
  out[x] = s;
}

// (f_hi, f_lo)[l][i][x] += c_l lam[x] gm[i][x]; with f_lo null a plain sum
// into f_hi, else a compensated pair (the rounding error of each add kept in f_lo)
template <typename T>
__global__ void k_force(T* __restrict__ fhi, T* __restrict__ flo, const T* __restrict__ lam,
                        const T* __restrict__ gm, Coefs c, int nc, int d, long N) {
  long x = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= N) return;
  T l = lam[x];
  for (int i = 0; i < d; ++i) {
    T p = l * gm[i * N + x];
    for (int a = 0; a < nc; ++a) {
      long q = ((long)a * d + i) * N + x;
      T t = (T)c.c[a] * p;
      if (!flo) {
        fhi[q] += t;
      } else {
        T h = fhi[q], sm = h + t, bp = sm - h;
        flo[q] += (h - (sm - bp)) + (t - bp);
        fhi[q] = sm;
      }
    }
  }
}

__global__ void k_pair_to_double(const float* __restrict__ hi, const float* __restrict__ lo, double* __restrict__ out,
                                 long n) {
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (double)hi[i] + (double)lo[i];
}

// det F right-hand side for component q = (a,c): -v.grad F_q + sum_m gv_{am} F_{mc}
__global__ void k_detF_rhs(const double* __restrict__ G, const double* __restrict__ vt,
                           const double* __restrict__ gv, const double* __restrict__ F, int q, double* __restrict__ k,
                           int d, long N) {
  long x = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= N) return;
  int a = q / d, c = q % d;
  double s = 0.0;
  for (int i = 0; i < d; ++i) s -= vt[i * N + x] * G[i * N + x];
  for (int m = 0; m < d; ++m) s += gv[(a * d + m) * N + x] * F[(m * d + c) * N + x];
  k[q * N + x] = s;
}

__global__ void k_identity_tensor(double* __restrict__ F, int d, long N) {
  long x = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= N) return;
  for (int a = 0; a < d; ++a)
    for (int c = 0; c < d; ++c) F[(a * d + c) * N + x] = (a == c) ? 1.0 : 0.0;
}

// per point, the smallest acute angle between two columns F e_c (deformed grid edges)
__global__ void k_grid_angle(const double* __restrict__ F, double* __restrict__ ang, int d, long N) {
  long x = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= N) return;
  const double half_pi = 1.5707963267948966;
  double best = half_pi;
  for (int c1 = 0; c1 < d; ++c1)
    for (int c2 = c1 + 1; c2 < d; ++c2) {
      double p = 0.0, n1 = 0.0, n2 = 0.0;
      for (int a = 0; a < d; ++a) {
        double f1 = F[(a * d + c1) * N + x], f2 = F[(a * d + c2) * N + x];
        p += f1 * f2;
        n1 += f1 * f1;
        n2 += f2 * f2;
      }
      double cs = fmin(1.0, fmax(-1.0, p / sqrt(n1 * n2)));
      double th = acos(cs);
      best = fmin(best, th < half_pi ? th : 2.0 * half_pi - th);
    }
  ang[x] = best;
}

__global__ void k_det(const double* __restrict__ F, double* __restrict__ det, int d, long N) {
  long x = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= N) return;
  if (d == 2) {
    det[x] = F[x] * F[3 * N + x] - F[N + x] * F[2 * N + x];
  } else {
    double a00 = F[x], a01 = F[N + x], a02 = F[2 * N + x];
    double a10 = F[3 * N + x], a11 = F[4 * N + x], a12 = F[5 * N + x];
    double a20 = F[6 * N + x], a21 = F[7 * N + x], a22 = F[8 * N + x];
    det[x] = a00 * (a11 * a22 - a12 * a21) - a01 * (a10 * a22 - a12 * a20) + a02 * (a10 * a21 - a11 * a20);
  }
}

template <typename T>
__global__ void k_lincomb_t(T a, const T* __restrict__ x, T b, const T* __restrict__ y, T* __restrict__ out, long n) {
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = a * x[i] + (y ? b * y[i] : (T)0);
}

__global__ void k_axpby(double a, const double* __restrict__ x, double b, double* __restrict__ y, long n) {
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = a * x[i] + b * y[i];
}

__global__ void k_lincomb(double a, const double* __restrict__ x, double b, const double* __restrict__ y,
                          double* __restrict__ out, long n) {
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = a * x[i] + b * y[i];
}

// ---------------------------------------------------------------------------
// Deterministic reductions: fixed grid, fixed per-thread striding, block tree
// in shared memory, then one block combines the partials in index order.
// ---------------------------------------------------------------------------
constexpr int kRedBlocks = 1024;
constexpr int kRedThreads = 256;

enum RedOp { RED_DOT = 0, RED_SQDIFF = 1, RED_MAXABS = 2, RED_STATS = 3 };

struct Acc4 {
  double s, s2, mn, mx;
};

template <int OP>
__global__ void k_reduce(const double* __restrict__ a, const double* __restrict__ b, long n, double center,
                         double* __restrict__ part) {
  __shared__ double sh[4][kRedThreads];
  double s = 0, s2 = 0, mn = DBL_MAX, mx = -DBL_MAX;
  for (long i = (long)blockIdx.x * kRedThreads + threadIdx.x; i < n; i += (long)kRedBlocks * kRedThreads) {
    double x = a[i];
    if (OP == RED_DOT) s += x * b[i];
    else if (OP == RED_SQDIFF) { double t = x - b[i]; s += t * t; }
    else if (OP == RED_MAXABS) mx = fmax(mx, fabs(x));
    else { double t = x - center; s += t; s2 += t * t; mn = fmin(mn, x); mx = fmax(mx, x); }
  }
  sh[0][threadIdx.x] = s;
  sh[1][threadIdx.x] = s2;
  sh[2][threadIdx.x] = mn;
  sh[3][threadIdx.x] = mx;
  __syncthreads();
  for (int w = kRedThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      sh[0][threadIdx.x] += sh[0][threadIdx.x + w];
      sh[1][threadIdx.x] += sh[1][threadIdx.x + w];
      sh[2][threadIdx.x] = fmin(sh[2][threadIdx.x], sh[2][threadIdx.x + w]);
      sh[3][threadIdx.x] = fmax(sh[3][threadIdx.x], sh[3][threadIdx.x + w]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int k = 0; k < 4; ++k) part[k * kRedBlocks + blockIdx.x] = sh[k][0];
}

__global__ void k_reduce_final(const double* __restrict__ part, double* __restrict__ out) {
  __shared__ double sh[4][kRedThreads];
  double s = 0, s2 = 0, mn = DBL_MAX, mx = -DBL_MAX;
  for (int i = threadIdx.x; i < kRedBlocks; i += kRedThreads) {
    s += part[i];
    s2 += part[kRedBlocks + i];
    mn = fmin(mn, part[2 * kRedBlocks + i]);
    mx = fmax(mx, part[3 * kRedBlocks + i]);
  }
  sh[0][threadIdx.x] = s;
  sh[1][threadIdx.x] = s2;
  sh[2][threadIdx.x] = mn;
  sh[3][threadIdx.x] = mx;
  __syncthreads();
  for (int w = kRedThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      sh[0][threadIdx.x] += sh[0][threadIdx.x + w];
      sh[1][threadIdx.x] += sh[1][threadIdx.x + w];
      sh[2][threadIdx.x] = fmin(sh[2][threadIdx.x], sh[2][threadIdx.x + w]);
      sh[3][threadIdx.x] = fmax(sh[3][threadIdx.x], sh[3][threadIdx.x + w]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int k = 0; k < 4; ++k) out[k] = sh[k][0];
}

}  // namespace

template <typename T, typename S>
void vel_at(const S* coef, int nc, const Coefs& b, T* out, long dN, cudaStream_t s) {
  k_vel_at<T, S><<<nblk(dN), 256, 0, s>>>(coef, nc, b, out, dN);
  REG_LAUNCH();
}
template void vel_at<float, double>(const double*, int, const Coefs&, float*, long, cudaStream_t);
template void vel_at<double, double>(const double*, int, const Coefs&, double*, long, cudaStream_t);
template void vel_at<float, float>(const float*, int, const Coefs&, float*, long, cudaStream_t);

template <typename S, typename T>
void convert(const S* in, T* out, long n, cudaStream_t s) {
  k_convert<S, T><<<nblk(n), 256, 0, s>>>(in, out, n);
  REG_LAUNCH();
}
template void convert<double, float>(const double*, float*, long, cudaStream_t);
template void convert<float, double>(const float*, double*, long, cudaStream_t);
template void convert<double, double>(const double*, double*, long, cudaStream_t);

template <typename T>
void transport_stage1(const T* G, const T* vt, const T* gm, const T* wt, const T* y, T h, T* yh, T* acc, int d,
                      long N, cudaStream_t s) {
  ProfScope ps(KK_STAGE, s, (double)N * sizeof(T) * ((G ? 2 * d : 0) + (gm ? 2 * d : 0) + (y ? 1 : 0) + 2));
  if (gm) k_stage<T, true, true><<<nblk(N), 256, 0, s>>>(G, vt, gm, wt, y, h, yh, acc, d, N);
  else k_stage<T, false, true><<<nblk(N), 256, 0, s>>>(G, vt, gm, wt, y, h, yh, acc, d, N);
  REG_LAUNCH();
}
template <typename T>
void dot_fields(const T* a, const T* b, T* out, int d, long N, cudaStream_t s) {
  ProfScope ps(KK_STAGE, s, (double)N * sizeof(T) * (2 * d + 1));
  k_dot_fields<T><<<nblk(N), 256, 0, s>>>(a, b, out, d, N);
  REG_LAUNCH();
}

template <typename T>
void force_acc(T* fhi, T* flo, const T* lam, const T* gm, const Coefs& c, int nc, int d, long N, cudaStream_t s) {
  ProfScope ps(KK_FORCE, s, (double)N * sizeof(T) * ((d + 1) + 2.0 * nc * d * (flo ? 2 : 1)));
  k_force<T><<<nblk(N), 256, 0, s>>>(fhi, flo, lam, gm, c, nc, d, N);
  REG_LAUNCH();
}

void pair_to_double(const float* hi, const float* lo, double* out, long n, cudaStream_t s) {
  k_pair_to_double<<<nblk(n), 256, 0, s>>>(hi, lo, out, n);
  REG_LAUNCH();
}

#define INST(T)                                                                                          \
  template void transport_stage1<T>(const T*, const T*, const T*, const T*, const T*, T, T*, T*, int, long, \
                                    cudaStream_t);                                                       \
  template void dot_fields<T>(const T*, const T*, T*, int, long, cudaStream_t);                             \
  template void force_acc<T>(T*, T*, const T*, const T*, const Coefs&, int, int, long, cudaStream_t);
INST(float)
INST(double)
#undef INST

template <typename T>
void lincomb_t(T a, const T* x, T b, const T* y, T* out, long n, cudaStream_t s) {
  k_lincomb_t<T><<<nblk(n), 256, 0, s>>>(a, x, b, y, out, n);
  REG_LAUNCH();
}
template void lincomb_t<float>(float, const float*, float, const float*, float*, long, cudaStream_t);
template void lincomb_t<double>(double, const double*, double, const double*, double*, long, cudaStream_t);

void detF_rhs(const double* G, const double* vt, const double* gv, const double* F, int q, double* k, int d, long N,
              cudaStream_t s) {
  k_detF_rhs<<<nblk(N), 256, 0, s>>>(G, vt, gv, F, q, k, d, N);
  REG_LAUNCH();
}
void identity_tensor(double* F, int d, long N, cudaStream_t s) {
  k_identity_tensor<<<nblk(N), 256, 0, s>>>(F, d, N);
  REG_LAUNCH();
}
void det_tensor(const double* F, double* det, int d, long N, cudaStream_t s) {
  k_det<<<nblk(N), 256, 0, s>>>(F, det, d, N);
  REG_LAUNCH();
}
void grid_angle_tensor(const double* F, double* angle, int d, long N, cudaStream_t s) {
  k_grid_angle<<<nblk(N), 256, 0, s>>>(F, angle, d, N);
  REG_LAUNCH();
}
void axpby(double a, const double* x, double b, double* y, long n, cudaStream_t s) {
  k_axpby<<<nblk(n), 256, 0, s>>>(a, x, b, y, n);
  REG_LAUNCH();
}
void lincomb(double a, const double* x, double b, const double* y, double* out, long n, cudaStream_t s) {
  k_lincomb<<<nblk(n), 256, 0, s>>>(a, x, b, y, out, n);
  REG_LAUNCH();
}

long reduce_scratch_doubles() { return 4L * kRedBlocks + 4; }

// ---------------------------------------------------------------------------
// Per-problem reductions and vector updates of B stacked problems: a vector
// of K components is laid out [K][B][N1]; problem p owns the slices
// [k][p][0..N1). Deterministic: fixed partial sums per (problem, block).
// ---------------------------------------------------------------------------
template <int OP>
__global__ void k_seg_reduce(const double* __restrict__ a, const double* __restrict__ b, int K, int B, long N1,
                             int nb, double* __restrict__ part) {
  __shared__ double sh[kRedThreads];
  const int p = blockIdx.y;
  double acc = 0.0;
  for (int k = 0; k < K; ++k) {
    const long base = ((long)k * B + p) * N1;
    for (long x = (long)blockIdx.x * kRedThreads + threadIdx.x; x < N1; x += (long)nb * kRedThreads) {
      const double u = a[base + x];
      if (OP == RED_DOT) acc += u * b[base + x];
      else if (OP == RED_SQDIFF) { double t = u - b[base + x]; acc += t * t; }
      else acc = fmax(acc, fabs(u));
    }
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int w = kRedThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      sh[threadIdx.x] = OP == RED_MAXABS ? fmax(sh[threadIdx.x], sh[threadIdx.x + w]) : sh[threadIdx.x] + sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[(long)p * nb + blockIdx.x] = sh[0];
}

__global__ void k_seg_final(const double* __restrict__ part, int nb, int B, int is_max, double* __restrict__ out) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= B) return;
  double acc = 0.0;
  for (int j = 0; j < nb; ++j) acc = is_max ? fmax(acc, part[(long)p * nb + j]) : acc + part[(long)p * nb + j];
  out[p] = acc;
}

// y = a_p x + c_p y per problem p (a zero coefficient drops its term, so a
// masked problem's values never enter, whatever they hold)
// grid: (ceil(N1 / blockDim), K * B); slice blockIdx.y is component / problem (k, p)
__global__ void k_axpby_seg(const double* __restrict__ a, const double* __restrict__ x,
                            const double* __restrict__ c, const double* y, double* out, int B, long N1, int y0) {
  const long xi = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (xi >= N1) return;
  const int slice = blockIdx.y + y0;
  const int p = slice % B;
  const long i = (long)slice * N1 + xi;
  const double ap = a[p], cp = c[p];
  out[i] = (ap != 0.0 ? ap * x[i] : 0.0) + (cp != 0.0 ? cp * y[i] : 0.0);
}

long seg_scratch_doubles(int B) { return (long)B * 32 + B; }

void seg_reduce(int op, const double* a, const double* b, int K, int B, long N1, double* scratch, cudaStream_t s,
                double* out_host) {
  if (B > 65535) throw StatusError{1, "more than 65535 stacked problems"};
  int nb = (int)(((long)K * N1 + 8L * kRedThreads - 1) / (8L * kRedThreads));
  nb = nb < 1 ? 1 : (nb > 32 ? 32 : nb);
  dim3 grid((unsigned)nb, (unsigned)B);
  switch (op) {
    case RED_DOT: k_seg_reduce<RED_DOT><<<grid, kRedThreads, 0, s>>>(a, b, K, B, N1, nb, scratch); break;
    case RED_SQDIFF: k_seg_reduce<RED_SQDIFF><<<grid, kRedThreads, 0, s>>>(a, b, K, B, N1, nb, scratch); break;
    default: k_seg_reduce<RED_MAXABS><<<grid, kRedThreads, 0, s>>>(a, b, K, B, N1, nb, scratch); break;
  }
  REG_LAUNCH();
  double* out = scratch + (long)B * 32;
  k_seg_final<<<(B + 127) / 128, 128, 0, s>>>(scratch, nb, B, op == RED_MAXABS, out);
  REG_LAUNCH();
  REG_CUDA(cudaMemcpyAsync(out_host, out, sizeof(double) * B, cudaMemcpyDeviceToHost, s));
  REG_CUDA(cudaStreamSynchronize(s));
}

void seg_reduce_dev(int op, const double* a, const double* b, int K, int B, long N1, double* scratch, cudaStream_t s,
                    double* out_dev) {
  if (B > 65535) throw StatusError{1, "more than 65535 stacked problems"};
  int nb = (int)(((long)K * N1 + 8L * kRedThreads - 1) / (8L * kRedThreads));  // as seg_reduce: the same sums
  nb = nb < 1 ? 1 : (nb > 32 ? 32 : nb);
  dim3 grid((unsigned)nb, (unsigned)B);
  switch (op) {
    case RED_DOT: k_seg_reduce<RED_DOT><<<grid, kRedThreads, 0, s>>>(a, b, K, B, N1, nb, scratch); break;
    default: k_seg_reduce<RED_SQDIFF><<<grid, kRedThreads, 0, s>>>(a, b, K, B, N1, nb, scratch); break;
  }
  REG_LAUNCH();
  k_seg_final<<<(B + 127) / 128, 128, 0, s>>>(scratch, nb, B, 0, out_dev);
  REG_LAUNCH();
}
void seg_dot_dev(const double* a, const double* b, int K, int B, long N1, double* scratch, cudaStream_t s,
                 double* out_dev) {
  seg_reduce_dev(RED_DOT, a, b, K, B, N1, scratch, s, out_dev);
}
void seg_sqdiff_dev(const double* a, const double* b, int K, int B, long N1, double* scratch, cudaStream_t s,
                    double* out_dev) {
  seg_reduce_dev(RED_SQDIFF, a, b, K, B, N1, scratch, s, out_dev);
}

// ---------------------------------------------------------------------------
// device-driven lockstep loops: one block of kLkThreads threads walks the B
// problems; the handles are set by thread 0 after a block-wide OR
// ---------------------------------------------------------------------------
constexpr int kLkThreads = 256;
#define LK(slot, q) lk[(long)(slot) * B + (q)]

__global__ void k_lk_pcg_init(double* lk, int* ctl, int B) {
  for (int q = threadIdx.x; q < B; q += blockDim.x) {
    LK(LK_ONE, q) = 1.0;
    LK(LK_ZERO, q) = 0.0;
    LK(LK_MONE, q) = -1.0;
    LK(LK_ON, q) = LK(LK_ACT, q);
    LK(LK_ETA, q) = fmin(0.5, sqrt(LK(LK_G2, q) / LK(LK_G02, q)));
    LK(LK_NEGC, q) = 0.0;
    LK(LK_KEEP, q) = 1.0;
    LK(LK_PCG, q) = LK(LK_MV, q) = LK(LK_NPDE, q) = LK(LK_LS, q) = 0.0;
    LK(LK_STATUS, q) = 0.0;
  }
  if (threadIdx.x < LC_COUNT) ctl[threadIdx.x] = 0;
}

__global__ void k_lk_pcg_check(double* lk, int* ctl, int B, int cap, int maxit, cudaGraphConditionalHandle h_if,
                               cudaGraphConditionalHandle h_while) {
  int any = 0;
  for (int q = threadIdx.x; q < B; q += blockDim.x) {
    if (LK(LK_ON, q) == 0.0) continue;
    const double rn2 = LK(LK_RN2, q);
    if (LK(LK_ACT, q) != 0.0 && !isfinite(rn2)) {
      LK(LK_ACT, q) = 0.0;
      LK(LK_STATUS, q) = 5.0;  // REG_ENONFINITE
    }
    if (LK(LK_ACT, q) == 0.0 || sqrt(rn2) <= __dmul_rn(LK(LK_ETA, q), LK(LK_G2, q))) LK(LK_ON, q) = 0.0;
    else any = 1;
  }
  any = __syncthreads_or(any);
  if (threadIdx.x == 0) {
    const int it = ctl[LC_IT];
    const int run = any && ctl[LC_PIT] < maxit;
    ctl[LC_ON] = any;
    if (run) ctl[LC_IT] = it + 1;
    cudaGraphSetConditional(h_if, run ? 1u : 0u);
    cudaGraphSetConditional(h_while, (run && it + 1 < cap) ? 1u : 0u);
  }
}

__global__ void k_lk_pcg_alpha(double* lk, int* ctl, int B) {
  const int pit = ctl[LC_PIT];
  for (int q = threadIdx.x; q < B; q += blockDim.x) {
    double a = 0.0, negc = 0.0;
    if (LK(LK_ON, q) != 0.0) {
      LK(LK_MV, q) += 1.0;
      LK(LK_NPDE, q) += 2.0;
      LK(LK_PCG, q) += 1.0;
      const double php = LK(LK_PHP, q);
      if (LK(LK_ACT, q) != 0.0 && !isfinite(php)) {
        LK(LK_ACT, q) = 0.0;
        LK(LK_STATUS, q) = 5.0;
      }
      if (LK(LK_ACT, q) == 0.0) {
        LK(LK_ON, q) = 0.0;
      } else if (php <= 0.0) {
        if (pit == 0) negc = 1.0;  // the steepest-descent direction
        LK(LK_ON, q) = 0.0;
      } else {
        a = LK(LK_RZ, q) / php;
      }
    }
    LK(LK_A, q) = a;
    LK(LK_NEGC, q) = negc;
    LK(LK_KEEP, q) = 1.0 - negc;
  }
}

__global__ void k_lk_pcg_beta(double* lk, int* ctl, int B) {
  for (int q = threadIdx.x; q < B; q += blockDim.x) {
    double mz = 0.0, bt = 1.0;
    if (LK(LK_ON, q) != 0.0) {
      mz = -1.0;
      bt = LK(LK_RZN, q) / LK(LK_RZ, q);
      LK(LK_RZ, q) = LK(LK_RZN, q);
    }
    LK(LK_MZ, q) = mz;
    LK(LK_BT, q) = bt;
  }
  if (threadIdx.x == 0) ctl[LC_PIT] += 1;
}

__global__ void k_lk_ls_init(double* lk, int* ctl, int B, double hd) {
  for (int q = threadIdx.x; q < B; q += blockDim.x) {
    LK(LK_SLOPE, q) = __dmul_rn(LK(LK_SLOPE, q), hd);
    const bool act = LK(LK_ACT, q) != 0.0;
    LK(LK_ALPHA, q) = act ? 1.0 : 0.0;
    LK(LK_SRCH, q) = act ? 1.0 : 0.0;
  }
  if (threadIdx.x == 0) ctl[LC_LST] = 0;
}

__global__ void k_lk_ls_check(double* lk, int* ctl, int B, int max_bt, cudaGraphConditionalHandle h_if,
                              cudaGraphConditionalHandle h_while) {
  int any = 0;
  for (int q = threadIdx.x; q < B; q += blockDim.x)
    if (LK(LK_SRCH, q) != 0.0) any = 1;
  any = __syncthreads_or(any);
  if (threadIdx.x == 0) {
    const int t = ctl[LC_LST];
    const int run = any && t < max_bt;
    if (run) ctl[LC_LST] = t + 1;
    cudaGraphSetConditional(h_if, run ? 1u : 0u);
    cudaGraphSetConditional(h_while, run ? 1u : 0u);
  }
}

__global__ void k_lk_ls_armijo(double* lk, int B, double hd, double c1, double rho) {
  for (int q = threadIdx.x; q < B; q += blockDim.x) {
    if (LK(LK_SRCH, q) == 0.0) continue;
    LK(LK_LS, q) += 1.0;
    LK(LK_NPDE, q) += 1.0;
    // J_t = 1/2 h_d d2 + 1/2 h_d r2, each part scaled as the host scales it
    const double half_hd = __dmul_rn(0.5, hd);
    const double jt = __dadd_rn(__dmul_rn(LK(LK_D2, q), half_hd), __dmul_rn(LK(LK_R2, q), half_hd));
    LK(LK_JT, q) = jt;
    const double a = LK(LK_ALPHA, q);
    const double bound = __dadd_rn(LK(LK_J, q), __dmul_rn(__dmul_rn(c1, a), LK(LK_SLOPE, q)));
    if (isfinite(jt) && jt <= bound) LK(LK_SRCH, q) = 0.0;
    else LK(LK_ALPHA, q) = __dmul_rn(a, rho);
  }
}

__global__ void k_lk_ls_final(double* lk, int B, int status_ls) {
  for (int q = threadIdx.x; q < B; q += blockDim.x) {
    if (LK(LK_SRCH, q) != 0.0) {
      LK(LK_ACT, q) = 0.0;
      LK(LK_STATUS, q) = (double)status_ls;
      LK(LK_ALPHA, q) = 0.0;
    }
    if (LK(LK_ACT, q) == 0.0) LK(LK_ALPHA, q) = 0.0;
  }
}
#undef LK

void lk_pcg_init(double* lk, int* ctl, int B, cudaStream_t s) {
  k_lk_pcg_init<<<1, kLkThreads, 0, s>>>(lk, ctl, B);
  REG_LAUNCH();
}
void lk_pcg_check(double* lk, int* ctl, int B, int cap, int maxit, unsigned long long h_if,
                  unsigned long long h_while, cudaStream_t s) {
  k_lk_pcg_check<<<1, kLkThreads, 0, s>>>(lk, ctl, B, cap, maxit, (cudaGraphConditionalHandle)h_if,
                                          (cudaGraphConditionalHandle)h_while);
  REG_LAUNCH();
}
void lk_pcg_alpha(double* lk, int* ctl, int B, cudaStream_t s) {
  k_lk_pcg_alpha<<<1, kLkThreads, 0, s>>>(lk, ctl, B);
  REG_LAUNCH();
}
void lk_pcg_beta(double* lk, int* ctl, int B, cudaStream_t s) {
  k_lk_pcg_beta<<<1, kLkThreads, 0, s>>>(lk, ctl, B);
  REG_LAUNCH();
}
void lk_ls_init(double* lk, int* ctl, int B, double hd, cudaStream_t s) {
  k_lk_ls_init<<<1, kLkThreads, 0, s>>>(lk, ctl, B, hd);
  REG_LAUNCH();
}
void lk_ls_check(double* lk, int* ctl, int B, int max_bt, unsigned long long h_if, unsigned long long h_while,
                 cudaStream_t s) {
  k_lk_ls_check<<<1, kLkThreads, 0, s>>>(lk, ctl, B, max_bt, (cudaGraphConditionalHandle)h_if,
                                         (cudaGraphConditionalHandle)h_while);
  REG_LAUNCH();
}
void lk_ls_armijo(double* lk, int B, double hd, double c1, double rho, cudaStream_t s) {
  k_lk_ls_armijo<<<1, kLkThreads, 0, s>>>(lk, B, hd, c1, rho);
  REG_LAUNCH();
}
void lk_ls_final(double* lk, int B, int status_ls, cudaStream_t s) {
  k_lk_ls_final<<<1, kLkThreads, 0, s>>>(lk, B, status_ls);
  REG_LAUNCH();
}

void seg_dot(const double* a, const double* b, int K, int B, long N1, double* scratch, cudaStream_t s, double* out) {
  seg_reduce(RED_DOT, a, b, K, B, N1, scratch, s, out);
}
void seg_sqdiff(const double* a, const double* b, int K, int B, long N1, double* scratch, cudaStream_t s,
                double* out) {
  seg_reduce(RED_SQDIFF, a, b, K, B, N1, scratch, s, out);
}
void seg_maxabs(const double* a, int K, int B, long N1, double* scratch, cudaStream_t s, double* out) {
  seg_reduce(RED_MAXABS, a, nullptr, K, B, N1, scratch, s, out);
}
void lincomb_seg(const double* a_dev, const double* x, const double* c_dev, const double* y, double* out, int K,
                 int B, long N1, cudaStream_t s) {
  for (int y0 = 0; y0 < K * B; y0 += 65535) {  // grid.y is limited to 65535 slices per launch
    const int ny = K * B - y0 < 65535 ? K * B - y0 : 65535;
    dim3 grid(nblk(N1), (unsigned)ny);
    k_axpby_seg<<<grid, 256, 0, s>>>(a_dev, x, c_dev, y, out, B, N1, y0);
    REG_LAUNCH();
  }
}

// result (device, 4 doubles at scratch + 4*kRedBlocks): {sum, sumsq, min, max}
static double* launch_reduce(int op, const double* a, const double* b, long n, double* scratch, cudaStream_t s,
                             double center = 0.0) {
  double* out = scratch + 4L * kRedBlocks;
  switch (op) {
    case RED_DOT: k_reduce<RED_DOT><<<kRedBlocks, kRedThreads, 0, s>>>(a, b, n, 0.0, scratch); break;
    case RED_SQDIFF: k_reduce<RED_SQDIFF><<<kRedBlocks, kRedThreads, 0, s>>>(a, b, n, 0.0, scratch); break;
    case RED_MAXABS: k_reduce<RED_MAXABS><<<kRedBlocks, kRedThreads, 0, s>>>(a, b, n, 0.0, scratch); break;
    default: k_reduce<RED_STATS><<<kRedBlocks, kRedThreads, 0, s>>>(a, b, n, center, scratch); break;
  }
  REG_LAUNCH();
  k_reduce_final<<<1, kRedThreads, 0, s>>>(scratch, out);
  REG_LAUNCH();
  return out;
}

static void fetch(const double* dev, double* host, int count, cudaStream_t s) {
  REG_CUDA(cudaMemcpyAsync(host, dev, sizeof(double) * count, cudaMemcpyDeviceToHost, s));
  REG_CUDA(cudaStreamSynchronize(s));
}

double dot(const double* a, const double* b, long n, double* scratch, cudaStream_t s) {
  double r[4];
  fetch(launch_reduce(RED_DOT, a, b, n, scratch, s), r, 4, s);
  return r[0];
}
double sqdiff(const double* a, const double* b, long n, double* scratch, cudaStream_t s) {
  double r[4];
  fetch(launch_reduce(RED_SQDIFF, a, b, n, scratch, s), r, 4, s);
  return r[0];
}
double maxabs(const double* a, long n, double* scratch, cudaStream_t s) {
  double r[4];
  fetch(launch_reduce(RED_MAXABS, a, nullptr, n, scratch, s), r, 4, s);
  return r[3];
}
// {min, max, mean, std}: two passes, the second centred on the mean
void stats(const double* a, long n, double* scratch, cudaStream_t s, double out[4]) {
  double r[4];
  fetch(launch_reduce(RED_STATS, a, nullptr, n, scratch, s, 0.0), r, 4, s);
  double mean = r[0] / n;
  fetch(launch_reduce(RED_STATS, a, nullptr, n, scratch, s, mean), r, 4, s);
  double c = r[0] / n;
  double var = r[1] / n - c * c;
  out[0] = r[2];
  out[1] = r[3];
  out[2] = mean + c;
  out[3] = var > 0 ? sqrt(var) : 0.0;
}

}  // namespace reg
