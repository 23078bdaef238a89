// spectral.cu -- FFT passes and Fourier multipliers of the pseudospectral
// discretisation (Mang & Biros, Sec. 3.3.1 Fourier collocation; Sec. 3.3.3 the
// spectral inverse of beta*A; Sec. 3.3.4 / App. B the Leray projection K).
//
// A d-dimensional real transform is one row pass (packed real-to-complex
// along the contiguous last axis) followed by one strided complex pass per
// remaining axis. The packed layout stores the DC and Nyquist columns of the
// last axis together in slot 0 (see Grid in internal.h); derivative and
// Leray multipliers treat both halves alike (their last-axis wavenumber is 0
// for both), while multipliers depending on |k| (A and its inverse) pair the
// mode k' with -k' to act on the two halves separately.
#include <math.h>

#include <algorithm>
#include <atomic>
#include <stdexcept>

#include "internal.h"

namespace reg {

namespace {

constexpr int kThreads = 256;

__host__ __device__ inline long kfull(long j, long n) { return j < n / 2 ? j : j - n; }
__host__ __device__ inline long kmask(long j, long n) { return j == n / 2 ? 0 : kfull(j, n); }

// ---------------------------------------------------------------------------
// Row pass: real rows of length L -> packed complex rows of M = L/2.
// A real row read as M complex values z_j = x_{2j} + i x_{2j+1} is transformed
// by an M-point FFT Z; then X_k = E_k + W_L^k O_k with E = (Z_k + conj Z_{M-k})/2,
// O = (Z_k - conj Z_{M-k})/(2i). Slot 0 receives X_0 + i X_M.
// ---------------------------------------------------------------------------
template <typename T, int L, int RB>
__global__ void __launch_bounds__(kThreads) k_rows_r2c(const T* __restrict__ in, cx<T>* __restrict__ out, long nrows,
                                                        const cx<T>* __restrict__ tw,
                                                        const cx<T>* __restrict__ twrc) {
  using C = cx<T>;
  constexpr int M = L / 2;
  constexpr int RS = padded_len(M);
  __shared__ C buf[RB * RS];
  const long row0 = (long)blockIdx.x * RB;
  const C* src = reinterpret_cast<const C*>(in);
  for (int e = threadIdx.x; e < RB * M; e += kThreads) {
    int r = e / M, j = e % M;
    long row = row0 + r;
    C z = mk<C>(0, 0);
    if (row < nrows) z = src[row * M + j];
    buf[r * RS + pad16(j)] = z;
  }
  __syncthreads();
  smem_fft<T, M, false, kThreads, RB>(buf, RS, tw);
  constexpr int H = M / 2 + 1;
  for (int e = threadIdx.x; e < RB * H; e += kThreads) {
    int r = e / H, k = e % H;
    long row = row0 + r;
    if (row >= nrows) continue;
    C* o = out + row * M;
    if (k == 0) {
      C z0 = buf[r * RS];
      o[0] = mk<C>(z0.x + z0.y, z0.x - z0.y);
    } else {
      C zk = buf[r * RS + pad16(k)], zm = buf[r * RS + pad16(M - k)];
      C E = cscale(cadd(zk, cconj(zm)), (T)0.5);
      C Od = cscale(cmul_mi(csub(zk, cconj(zm))), (T)0.5);
      C t = cmul(__ldg(&twrc[k]), Od);
      o[k] = cadd(E, t);
      if (k != M - k) o[M - k] = cconj(csub(E, t));
    }
  }
}

// Inverse of the row pass, normalised by 1/L.
template <typename T, int L, int RB>
__global__ void __launch_bounds__(kThreads) k_rows_c2r(const cx<T>* __restrict__ in, T* __restrict__ out, long nrows,
                                                        const cx<T>* __restrict__ tw,
                                                        const cx<T>* __restrict__ twrc) {
  using C = cx<T>;
  constexpr int M = L / 2;
  constexpr int RS = padded_len(M);
  __shared__ C buf[RB * RS];
  const long row0 = (long)blockIdx.x * RB;
  for (int e = threadIdx.x; e < RB * M; e += kThreads) {
    int r = e / M, j = e % M;
    long row = row0 + r;
    C z = mk<C>(0, 0);
    if (row < nrows) z = in[row * M + j];
    buf[r * RS + pad16(j)] = z;
  }
  __syncthreads();
  constexpr int H = M / 2 + 1;
  for (int e = threadIdx.x; e < RB * H; e += kThreads) {
    int r = e / H, k = e % H;
    if (k == 0) {
      C p = buf[r * RS];
      // X_0 = p.x, X_M = p.y; E_0 = (X_0+X_M)/2, O_0 = (X_0-X_M)/2
      C z0 = mk<C>((p.x + p.y) * (T)0.5, (p.x - p.y) * (T)0.5);
      buf[r * RS] = cconj(z0);
    } else {
      C xk = buf[r * RS + pad16(k)], xm = buf[r * RS + pad16(M - k)];
      C E = cscale(cadd(xk, cconj(xm)), (T)0.5);
      C Od = cscale(cmul(csub(xk, cconj(xm)), cconj(__ldg(&twrc[k]))), (T)0.5);
      // Z_k = E + i O, Z_{M-k} = conj(E) + i conj(O); stored conjugated for the inverse
      C zk = mk<C>(E.x - Od.y, E.y + Od.x);
      C zm = mk<C>(E.x + Od.y, -E.y + Od.x);
      buf[r * RS + pad16(k)] = cconj(zk);
      if (k != M - k) buf[r * RS + pad16(M - k)] = cconj(zm);
    }
  }
  __syncthreads();
  smem_fft<T, M, false, kThreads, RB>(buf, RS, tw);
  C* dst = reinterpret_cast<C*>(out);
  const T s = (T)1 / (T)M;
  for (int e = threadIdx.x; e < RB * M; e += kThreads) {
    int r = e / M, j = e % M;
    long row = row0 + r;
    if (row >= nrows) continue;
    C z = buf[r * RS + pad16(j)];
    dst[row * M + j] = mk<C>(z.x * s, -z.y * s);
  }
}

// Strided complex pass along one axis: element j of pencil (outer, inner) at
// data[outer*L*s + j*s + inner]. A block takes TC neighbouring inner indices.
template <typename T, int L, int TC>
__global__ void __launch_bounds__(kThreads) k_cols(cx<T>* __restrict__ data, long s, const cx<T>* __restrict__ tw,
                                                    int inverse) {
  using C = cx<T>;
  __shared__ C buf[L * TC];
  C* base = data + (long)blockIdx.y * L * s + (long)blockIdx.x * TC;
  for (int e = threadIdx.x; e < L * TC; e += kThreads) {
    int j = e / TC, c = e % TC;
    C z = base[(long)j * s + c];
    buf[j * TC + c] = inverse ? cconj(z) : z;
  }
  __syncthreads();
  smem_fft<T, L, true, kThreads, TC>(buf, TC, tw);
  const T sc = (T)1 / (T)L;
  for (int e = threadIdx.x; e < L * TC; e += kThreads) {
    int j = e / TC, c = e % TC;
    C z = buf[j * TC + c];
    base[(long)j * s + c] = inverse ? mk<C>(z.x * sc, -z.y * sc) : z;
  }
}

// mode index q of the packed spectrum -> per-axis indices (last = slot)
struct ModeIdx {
  long j[3];
};
__device__ inline ModeIdx decode(long q, int d, const int* n, int M) {
  ModeIdx m;
  m.j[d - 1] = q % M;
  long rest = q / M;
  for (int a = d - 2; a >= 0; --a) {
    m.j[a] = rest % n[a];
    rest /= n[a];
  }
  return m;
}
struct GridArgs {
  int d;
  int n[3];
  int M;
  long Nc;   // all stacked problems
  long Nc1;  // one problem
};
// index of -k' on the slot-0 plane of the problem that holds mode q
__device__ inline long encode_neg(long q0, const ModeIdx& m, const GridArgs& g) {
  long q = 0;
  for (int a = 0; a < g.d - 1; ++a) q = q * g.n[a] + ((g.n[a] - m.j[a]) % g.n[a]);
  return (q0 / g.Nc1) * g.Nc1 + q * g.M;
}
__device__ inline double masked_k(const ModeIdx& m, const GridArgs& g, int a) {
  if (a == g.d - 1) return (double)m.j[a];  // slot 0 -> 0 for both DC and Nyquist halves
  return (double)kmask(m.j[a], g.n[a]);
}

template <typename T>
__global__ void k_mult_deriv(const cx<T>* __restrict__ U, cx<T>* __restrict__ W, GridArgs g, int axis, int acc) {
  long q = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= g.Nc) return;
  ModeIdx m = decode(q, g.d, g.n, g.M);
  T k = (T)masked_k(m, g, axis);
  cx<T> u = U[q];
  cx<T> r = mk<cx<T>>(-k * u.y, k * u.x);
  if (acc) r = cadd(W[q], r);
  W[q] = r;
}

template <typename T>
__global__ void k_mult_leray(cx<T>* __restrict__ W, GridArgs g) {
  long q = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= g.Nc) return;
  ModeIdx m = decode(q, g.d, g.n, g.M);
  T k[3];
  T kk = 0;
  for (int a = 0; a < g.d; ++a) {
    k[a] = (T)masked_k(m, g, a);
    kk += k[a] * k[a];
  }
  if (kk == (T)0) return;
  T dr = 0, di = 0;
  for (int a = 0; a < g.d; ++a) {
    cx<T> w = W[a * g.Nc + q];
    dr += k[a] * w.x;
    di += k[a] * w.y;
  }
  for (int a = 0; a < g.d; ++a) {
    cx<T> w = W[a * g.Nc + q];
    W[a * g.Nc + q] = mk<cx<T>>(w.x - k[a] * dr / kk, w.y - k[a] * di / kk);
  }
}

// |k|^2 over the leading axes (full wavenumbers, Nyquist kept)
__device__ inline double lead_k2(const ModeIdx& m, const GridArgs& g) {
  double kk = 0;
  for (int a = 0; a < g.d - 1; ++a) {
    double k = (double)kfull(m.j[a], g.n[a]);
    kk += k * k;
  }
  return kk;
}
__device__ inline double sym_pow(double kk, int reg) { return reg == 1 ? kk : kk * kk; }

constexpr int kMaxNc = 16;

__global__ void k_spec_tail(const double2* __restrict__ V, const double2* __restrict__ F, double2* __restrict__ out,
                            GridArgs g, int nc, double beta, const double* __restrict__ Cg, int reg, int stokes,
                            const double* __restrict__ betas) {
  long q = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= g.Nc) return;
  if (betas) beta = betas[q / g.Nc1];
  const int d = g.d;
  const long Nc = g.Nc;
  ModeIdx m = decode(q, d, g.n, g.M);
  double kk = lead_k2(m, g);
  long kz = m.j[d - 1];
  double alpha, delta;
  long qn = q;
  if (kz == 0) {
    double a0 = sym_pow(kk, reg), aN = sym_pow(kk + 0.25 * (double)g.n[d - 1] * g.n[d - 1], reg);
    alpha = 0.5 * (a0 + aN);
    delta = 0.5 * (a0 - aN);
    qn = encode_neg(q, m, g);
  } else {
    alpha = sym_pow(kk + (double)kz * kz, reg);
    delta = 0.0;
  }
  // masked wavenumber for K
  double kt[3], kt2 = 0;
  for (int a = 0; a < d; ++a) {
    kt[a] = masked_k(m, g, a);
    kt2 += kt[a] * kt[a];
  }
  for (int l = 0; l < nc; ++l) {
    double2 proj[3];
    if (F) {
      double dr = 0, di = 0;
      for (int i = 0; i < d; ++i) {
        double2 f = F[(l * d + i) * Nc + q];
        proj[i] = f;
        dr += kt[i] * f.x;
        di += kt[i] * f.y;
      }
      if (stokes && kt2 > 0)
        for (int i = 0; i < d; ++i) proj[i] = make_double2(proj[i].x - kt[i] * dr / kt2, proj[i].y - kt[i] * di / kt2);
    } else {
      for (int i = 0; i < d; ++i) proj[i] = make_double2(0, 0);
    }
    for (int i = 0; i < d; ++i) {
      double sr = 0, si = 0;
      for (int lp = 0; lp < nc; ++lp) {
        double c = Cg[l * nc + lp];
        double2 v = V[(lp * d + i) * Nc + q];
        double2 vn = V[(lp * d + i) * Nc + qn];
        // alpha v + delta conj(vn)
        sr += c * (alpha * v.x + delta * vn.x);
        si += c * (alpha * v.y - delta * vn.y);
      }
      out[(l * d + i) * Nc + q] = make_double2(beta * sr + proj[i].x, beta * si + proj[i].y);
    }
  }
}

__global__ void k_spec_precond(const double2* __restrict__ R, double2* __restrict__ out, GridArgs g, int nc,
                               double beta, const double* __restrict__ Ci, int reg, const double* __restrict__ betas) {
  long q = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= g.Nc) return;
  if (betas) beta = betas[q / g.Nc1];
  const int d = g.d;
  const long Nc = g.Nc;
  ModeIdx m = decode(q, d, g.n, g.M);
  double kk = lead_k2(m, g);
  long kz = m.j[d - 1];
  double alpha, delta;
  long qn = q;
  if (kz == 0) {
    double a0 = sym_pow(kk, reg), aN = sym_pow(kk + 0.25 * (double)g.n[d - 1] * g.n[d - 1], reg);
    double s0 = (q % g.Nc1 == 0) ? 1.0 : 1.0 / (beta * a0);  // k = 0: the inverse is replaced by one
    double sN = 1.0 / (beta * aN);
    alpha = 0.5 * (s0 + sN);
    delta = 0.5 * (s0 - sN);
    qn = encode_neg(q, m, g);
  } else {
    alpha = 1.0 / (beta * sym_pow(kk + (double)kz * kz, reg));
    delta = 0.0;
  }
  for (int l = 0; l < nc; ++l)
    for (int i = 0; i < d; ++i) {
      double sr = 0, si = 0;
      for (int lp = 0; lp < nc; ++lp) {
        double c = Ci[l * nc + lp];
        double2 v = R[(lp * d + i) * Nc + q];
        double2 vn = R[(lp * d + i) * Nc + qn];
        sr += c * (alpha * v.x + delta * vn.x);
        si += c * (alpha * v.y - delta * vn.y);
      }
      out[(l * d + i) * Nc + q] = make_double2(sr, si);
    }
}

// Gaussian filter exp(-sigma^2 |k|^2 / 2) on one packed field (full
// wavenumbers, Nyquist kept; slot 0 of the last axis pairs k' with -k' as A does)
__global__ void k_spec_gauss(double2* __restrict__ U, double2* __restrict__ out, GridArgs g, double s2) {
  long q = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= g.Nc) return;
  const int d = g.d;
  ModeIdx m = decode(q, d, g.n, g.M);
  double kk = lead_k2(m, g);
  long kz = m.j[d - 1];
  double2 v = U[q];
  if (kz == 0) {
    double g0 = exp(-0.5 * s2 * kk), gN = exp(-0.5 * s2 * (kk + 0.25 * (double)g.n[d - 1] * g.n[d - 1]));
    double alpha = 0.5 * (g0 + gN), delta = 0.5 * (g0 - gN);
    double2 vn = U[encode_neg(q, m, g)];
    out[q] = make_double2(alpha * v.x + delta * vn.x, alpha * v.y - delta * vn.y);
  } else {
    double gk = exp(-0.5 * s2 * (kk + (double)kz * kz));
    out[q] = make_double2(gk * v.x, gk * v.y);
  }
}

GridArgs args(const Grid& g) {
  GridArgs a;
  a.d = g.d;
  for (int i = 0; i < 3; ++i) a.n[i] = g.n[i];
  a.M = g.M;
  a.Nc = g.Nc;
  a.Nc1 = g.Nc / g.B;
  return a;
}

int ilog2(long n) {
  int e = 0;
  while ((1L << e) < n) ++e;
  return e;
}

// radix plan mirrored on the host (see Plan<> in fft.cuh)
std::vector<int> host_plan(int L) {
  switch (L) {
    case 2: return {2};
    case 4: return {4};
    case 8: return {8};
    case 16: return {16};
    case 32: return {8, 4};
    case 64: return {8, 8};
    case 128: return {16, 8};
    case 256: return {16, 16};
    case 512: return {8, 8, 8};
  }
  throw StatusError{1, "unsupported FFT length " + std::to_string(L)};
}

// Stage tables for length L: for stages s >= 1 (radix R, Ns previous), the
// entries W_{Ns R}^{r k} at [r*Ns + k], computed in double precision.
std::vector<double> stage_table(int L) {
  std::vector<double> t;
  std::vector<int> R = host_plan(L);
  int ns = R[0];
  for (size_t s = 1; s < R.size(); ++s) {
    for (int r = 0; r < R[s]; ++r)
      for (int k = 0; k < ns; ++k) {
        double ang = -2.0 * M_PI * (double)(r * k) / (double)(ns * R[s]);
        t.push_back(cos(ang));
        t.push_back(sin(ang));
      }
    ns *= R[s];
  }
  return t;
}

template <typename T, int L, int RB>
void launch_rows(bool inverse, const void* in, void* out, long nrows, const cx<T>* tw, const cx<T>* twrc,
                 cudaStream_t s) {
  ProfScope ps(inverse ? KK_ROWS_C2R : KK_ROWS_R2C, s, 2.0 * (double)nrows * L * sizeof(T),
               (double)nrows * (fft_flops<L / 2>() + 8.0 * (L / 2)));
  dim3 grid((unsigned)((nrows + RB - 1) / RB));
  if (!inverse)
    k_rows_r2c<T, L, RB><<<grid, kThreads, 0, s>>>((const T*)in, (cx<T>*)out, nrows, tw, twrc);
  else
    k_rows_c2r<T, L, RB><<<grid, kThreads, 0, s>>>((const cx<T>*)in, (T*)out, nrows, tw, twrc);
  REG_LAUNCH();
}

template <typename T>
void dispatch_rows(int L, bool inverse, const void* in, void* out, long nrows, const cx<T>* tw,
                   const cx<T>* twrc, cudaStream_t s) {
  // about 2048 (fp32) / 1024 (fp64) complex values per block
  constexpr int E = sizeof(T) == 4 ? 2048 : 1024;
  switch (L) {
    case 8: return launch_rows<T, 8, E / 4>(inverse, in, out, nrows, tw, twrc, s);
    case 16: return launch_rows<T, 16, E / 8>(inverse, in, out, nrows, tw, twrc, s);
    case 32: return launch_rows<T, 32, E / 16>(inverse, in, out, nrows, tw, twrc, s);
    case 64: return launch_rows<T, 64, E / 32>(inverse, in, out, nrows, tw, twrc, s);
    case 128: return launch_rows<T, 128, E / 64>(inverse, in, out, nrows, tw, twrc, s);
    case 256: return launch_rows<T, 256, E / 128>(inverse, in, out, nrows, tw, twrc, s);
    case 512: return launch_rows<T, 512, E / 256>(inverse, in, out, nrows, tw, twrc, s);
  }
  throw StatusError{1, "unsupported last-axis length " + std::to_string(L)};
}

template <typename T, int L, int TC>
void launch_cols(cx<T>* U, long s, long outer, const cx<T>* tw, bool inverse, cudaStream_t st) {
  ProfScope ps(KK_COLS, st, 2.0 * (double)s * outer * L * sizeof(cx<T>), (double)s * outer * fft_flops<L>());
  dim3 grid((unsigned)(s / TC), (unsigned)outer);
  k_cols<T, L, TC><<<grid, kThreads, 0, st>>>(U, s, tw, inverse ? 1 : 0);
  REG_LAUNCH();
}

template <typename T, int L>
void dispatch_cols_tc(cx<T>* U, long s, long outer, const cx<T>* tw, bool inverse, cudaStream_t st) {
  // tiles of 128-byte column segments (capped so the tile fits 32 KB)
  constexpr int TCmax0 = sizeof(T) == 4 ? 16 : 8;
  constexpr int TCmax = (L * TCmax0 * sizeof(cx<T>) > 32768) ? TCmax0 / 2 : TCmax0;
  if (s >= TCmax) return launch_cols<T, L, TCmax>(U, s, outer, tw, inverse, st);
  if (s >= 4) return launch_cols<T, L, 4>(U, s, outer, tw, inverse, st);
  return launch_cols<T, L, 2>(U, s, outer, tw, inverse, st);
}

template <typename T>
void dispatch_cols(int L, cx<T>* U, long s, long outer, const cx<T>* tw, bool inverse, cudaStream_t st) {
  switch (L) {
    case 8: return dispatch_cols_tc<T, 8>(U, s, outer, tw, inverse, st);
    case 16: return dispatch_cols_tc<T, 16>(U, s, outer, tw, inverse, st);
    case 32: return dispatch_cols_tc<T, 32>(U, s, outer, tw, inverse, st);
    case 64: return dispatch_cols_tc<T, 64>(U, s, outer, tw, inverse, st);
    case 128: return dispatch_cols_tc<T, 128>(U, s, outer, tw, inverse, st);
    case 256: return dispatch_cols_tc<T, 256>(U, s, outer, tw, inverse, st);
    case 512: return dispatch_cols_tc<T, 512>(U, s, outer, tw, inverse, st);
  }
  throw StatusError{1, "unsupported axis length " + std::to_string(L)};
}

unsigned blocks_for(long n, int bs = 256) { return (unsigned)((n + bs - 1) / bs); }

}  // namespace

Grid make_grid(int d, const int64_t* n, int batch) {
  Grid g;
  if (batch < 1) throw StatusError{1, "batch must be >= 1"};
  if (d != 2 && d != 3) throw StatusError{1, "d must be 2 or 3"};
  g.d = d;
  g.N = 1;
  for (int a = 0; a < d; ++a) {
    int64_t k = n[a];
    if (k < 8 || k > 512 || (k & (k - 1)) != 0)
      throw StatusError{1, "grid sizes must be powers of two in [8, 512]"};
    g.n[a] = (int)k;
    g.N *= k;
  }
  g.N1 = g.N;
  g.B = batch;
  g.N *= batch;
  g.L = g.n[d - 1];
  g.M = g.L / 2;
  g.Nc = g.N / 2;
  g.rows = g.N / g.L;
  return g;
}

template <typename T>
Spectral<T>::Spectral(const Grid& g, cudaStream_t s) : g_(g), s_(s) {
  // tables for every power of two from 4 to 512 (row half-length and axes)
  std::vector<double> all;
  for (int e = 2; e <= 9; ++e) {
    tw_off_[e] = (long)all.size() / 2;
    std::vector<double> t = stage_table(1 << e);
    all.insert(all.end(), t.begin(), t.end());
  }
  rc_off_ = (long)all.size() / 2;
  for (int k = 0; k < g.M; ++k) {
    double ang = -2.0 * M_PI * (double)k / (double)g.L;
    all.push_back(cos(ang));
    all.push_back(sin(ang));
  }
  std::vector<T> h(all.size());
  for (size_t i = 0; i < all.size(); ++i) h[i] = (T)all[i];
  REG_CUDA(cudaMalloc(&tw_, h.size() * sizeof(T)));
  REG_CUDA(cudaMemcpy(tw_, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
  if (sizeof(T) == 4) {
    // the two-stage plans' stage-1 blocks (L = 32..256) with duplicated entries
    std::vector<float4> p2;
    for (int e = 5; e <= 8; ++e) {
      tw2_off_[e] = (long)p2.size();
      std::vector<double> t = stage_table(1 << e);
      for (size_t i = 0; i + 1 < t.size(); i += 2)
        p2.push_back(make_float4((float)t[i], (float)t[i], (float)t[i + 1], (float)t[i + 1]));
    }
    REG_CUDA(cudaMalloc(&tw2_, p2.size() * sizeof(float4)));
    REG_CUDA(cudaMemcpy(tw2_, p2.data(), p2.size() * sizeof(float4), cudaMemcpyHostToDevice));
  }
}

template <typename T>
Spectral<T>::Spectral(const Grid& g, cudaStream_t s, C* tables, const long* tw_off, long rc_off)
    : g_(g), s_(s), tw_(tables), owns_(false) {
  for (int e = 0; e < 11; ++e) tw_off_[e] = tw_off[e];
  rc_off_ = rc_off;
}

template <typename T>
long Spectral<T>::write_tables(double* out, long* tw_off, long* rc_off) {
  long pos = 0;
  auto put = [&](double re, double im) {
    if (out) {
      out[2 * pos] = re;
      out[2 * pos + 1] = im;
    }
    ++pos;
  };
  for (int e = 0; e < 11; ++e) tw_off[e] = rc_off[e] = 0;
  for (int e = 2; e <= 9; ++e) {
    int L = 1 << e;
    tw_off[e] = pos;
    // the radix plan of Plan<L> (fft.cuh), in a fixed array: no heap use here
    int R[3] = {L, 1, 1}, S = 1;
    if (L == 32) { R[0] = 8; R[1] = 4; S = 2; }
    else if (L == 64) { R[0] = 8; R[1] = 8; S = 2; }
    else if (L == 128) { R[0] = 16; R[1] = 8; S = 2; }
    else if (L == 256) { R[0] = 16; R[1] = 16; S = 2; }
    else if (L == 512) { R[0] = 8; R[1] = 8; R[2] = 8; S = 3; }
    int ns = R[0];
    for (int st = 1; st < S; ++st) {
      for (int r = 0; r < R[st]; ++r)
        for (int k = 0; k < ns; ++k) {
          double ang = -2.0 * M_PI * (double)(r * k) / (double)(ns * R[st]);
          put(cos(ang), sin(ang));
        }
      ns *= R[st];
    }
  }
  for (int e = 3; e <= 9; ++e) {
    int L = 1 << e;
    rc_off[e] = pos;
    for (int k = 0; k < L / 2; ++k) {
      double ang = -2.0 * M_PI * (double)k / (double)L;
      put(cos(ang), sin(ang));
    }
  }
  return pos;
}

template <typename T>
Spectral<T>::~Spectral() {
  if (tw_ && owns_) cudaFree(tw_);
  if (tw2_ && owns_) cudaFree(tw2_);
  if (ev_fork_) cudaEventDestroy(ev_fork_);
  if (ev_join_) cudaEventDestroy(ev_join_);
  if (aux_) cudaStreamDestroy(aux_);
}

template <typename T>
cudaStream_t Spectral<T>::aux_stream() {
  if (!aux_) {
    REG_CUDA(cudaEventCreateWithFlags(&ev_fork_, cudaEventDisableTiming));
    REG_CUDA(cudaEventCreateWithFlags(&ev_join_, cudaEventDisableTiming));
    REG_CUDA(cudaStreamCreateWithFlags(&aux_, cudaStreamNonBlocking));
  }
  return aux_;
}

template <typename T>
const cx<T>* Spectral<T>::twiddles(int L) const {
  return tw_ + tw_off_[ilog2(L)];
}
template <typename T>
const cx<T>* Spectral<T>::rc_twiddles() const {
  return tw_ + rc_off_;
}
template <typename T>
const float4* Spectral<T>::pair_twiddles(int L) const {
  if (!tw2_ || L < 32 || L > 256) return nullptr;
  return tw2_ + tw2_off_[ilog2(L)];
}

template <typename T>
void Spectral<T>::cols(C* U, int axis, bool inverse) {
  long s = g_.M;
  for (int a = axis + 1; a < g_.d - 1; ++a) s *= g_.n[a];
  long outer = g_.Nc / (s * g_.n[axis]);
  dispatch_cols<T>(g_.n[axis], U, s, outer, twiddles(g_.n[axis]), inverse, s_);
}

template <typename T>
void Spectral<T>::fwd(const T* u, C* U) {
  dispatch_rows<T>(g_.L, false, u, U, g_.rows, twiddles(g_.M), rc_twiddles(), s_);
  for (int a = g_.d - 2; a >= 0; --a) cols(U, a, false);
}

template <typename T>
void Spectral<T>::inv(C* U, T* u) {
  for (int a = 0; a <= g_.d - 2; ++a) cols(U, a, true);
  dispatch_rows<T>(g_.L, true, U, u, g_.rows, twiddles(g_.M), rc_twiddles(), s_);
}

template <typename T>
void Spectral<T>::mult_deriv(const C* U, C* W, int axis) {
  ProfScope ps(KK_MULT, s_, 2.0 * g_.Nc * sizeof(C));
  k_mult_deriv<T><<<blocks_for(g_.Nc), 256, 0, s_>>>(U, W, args(g_), axis, 0);
  REG_LAUNCH();
}

template <typename T>
void Spectral<T>::mult_deriv_acc(const C* U, C* S, int axis, bool first) {
  ProfScope ps(KK_MULT, s_, (first ? 2.0 : 3.0) * g_.Nc * sizeof(C));
  k_mult_deriv<T><<<blocks_for(g_.Nc), 256, 0, s_>>>(U, S, args(g_), axis, first ? 0 : 1);
  REG_LAUNCH();
}

template <typename T>
void Spectral<T>::mult_leray(C* W) {
  k_mult_leray<T><<<blocks_for(g_.Nc), 256, 0, s_>>>(W, args(g_));
  REG_LAUNCH();
}

template <typename T>
void Spectral<T>::grad(const T* u, T* G, C* U, C* W) {
  fwd(u, U);
  for (int i = 0; i < g_.d; ++i) {
    mult_deriv(U, W, i);
    inv(W, G + (long)i * g_.N);
  }
}

template <typename T>
void Spectral<T>::div(const T* q, T* out, C* U, C* S) {
  for (int i = 0; i < g_.d; ++i) {
    fwd(q + (long)i * g_.N, U);
    mult_deriv_acc(U, S, i, i == 0);
  }
  inv(S, out);
}

template class Spectral<float>;

template class Spectral<double>;

void spec_tail(const Grid& g, cudaStream_t s, const double2* V, const double2* F, double2* out, int nc, double beta,
               const double* Cg_dev, int reg, int stokes, const double* betas) {
  if (nc > kMaxNc) throw StatusError{1, "n_c too large"};
  k_spec_tail<<<blocks_for(g.Nc), 256, 0, s>>>(V, F, out, args(g), nc, beta, Cg_dev, reg, stokes, betas);
  REG_LAUNCH();
}

void spec_precond(const Grid& g, cudaStream_t s, const double2* R, double2* out, int nc, double beta,
                  const double* Ci_dev, int reg, const double* betas) {
  k_spec_precond<<<blocks_for(g.Nc), 256, 0, s>>>(R, out, args(g), nc, beta, Ci_dev, reg, betas);
  REG_LAUNCH();
}

void spec_gauss(const Grid& g, cudaStream_t s, double2* U, double2* out, double sigma) {
  k_spec_gauss<<<blocks_for(g.Nc), 256, 0, s>>>(U, out, args(g), sigma * sigma);
  REG_LAUNCH();
}

// Trigonometric interpolation onto a grid refined per axis: the packed
// spectrum Q of the fine grid f from the packed spectrum P of the coarse grid
// c (nfields fields each; scale = N_f / N_c, so the fine inverse transform
// returns point values). A mode with |k_a| < n_a/2 on every axis keeps its
// coefficient; every other mode is zero, the coarse Nyquist modes included:
// the coarse derivatives treat those as constants (first derivatives and the
// Leray projection use the masked wavenumber), so the interpolated field is
// the part of the velocity that the coarse operators differentiate, and a
// velocity that is divergence-free on the coarse grid stays divergence-free.
// On the last axis the coarse slot 0 (DC + i Nyquist, both Hermitian in the
// other axes) is unpacked and its DC half goes to the fine slot 0.
__global__ void k_spec_upsample(const double2* __restrict__ P, double2* __restrict__ Q, GridArgs c, GridArgs f,
                                int nfields, double scale) {
  const long total = (long)nfields * f.Nc;
  for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
    const long fld = t / f.Nc, q = t % f.Nc;
    const ModeIdx m = decode(q, f.d, f.n, f.M);
    bool zero = m.j[f.d - 1] >= c.M;
    long row = 0, nrow = 0;  // coarse row of k' and of -k'
    for (int a = 0; a < f.d - 1 && !zero; ++a) {
      const long i = m.j[a];
      const long k = i < f.n[a] / 2 ? i : i - f.n[a];
      const long h = c.n[a] / 2;
      if (k >= h || k <= -h) {
        zero = true;
        break;
      }
      const long ci = (k + c.n[a]) % c.n[a];
      row = row * c.n[a] + ci;
      nrow = nrow * c.n[a] + (c.n[a] - ci) % c.n[a];
    }
    double2 out = make_double2(0.0, 0.0);
    if (!zero) {
      const double2* Pf = P + fld * c.Nc;
      const long kz = m.j[f.d - 1];
      if (kz > 0) {
        const double2 z = Pf[row * c.M + kz];
        out = make_double2(scale * z.x, scale * z.y);
      } else {  // the DC half of the coarse slot 0: (z + conj(zn)) / 2
        const double2 z = Pf[row * c.M], zn = Pf[nrow * c.M];
        out = make_double2(0.5 * scale * (z.x + zn.x), 0.5 * scale * (z.y - zn.y));
      }
    }
    Q[fld * f.Nc + q] = out;
  }
}

void spec_upsample(const Grid& c, const Grid& f, cudaStream_t s, const double2* P, double2* Q, int nfields) {
  const long total = (long)nfields * f.Nc;
  const int blocks = (int)std::min<long>((total + 255) / 256, 152L * 16);
  k_spec_upsample<<<blocks, 256, 0, s>>>(P, Q, args(c), args(f), nfields, (double)f.N / (double)c.N);
  REG_LAUNCH();
}

}  // namespace reg

namespace reg {

static std::atomic<long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void add_launches(long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long launch_count() { return g_launches.load(std::memory_order_relaxed); }

thread_local KernelProfiler* tl_prof = nullptr;

KernelProfiler::~KernelProfiler() {
  for (auto& r : recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (auto e : pool) cudaEventDestroy(e);
}

cudaEvent_t KernelProfiler::take() {
  if (!pool.empty()) {
    cudaEvent_t e = pool.back();
    pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  REG_CUDA(cudaEventCreate(&e));
  return e;
}

void KernelProfiler::collect(double* ms, double* bytes, long* count) {
  for (int k = 0; k < KK_COUNT; ++k) {
    ms[k] = 0;
    bytes[k] = 0;
    count[k] = 0;
    last_flops[k] = 0;
  }
  for (auto& r : recs) {
    REG_CUDA(cudaEventSynchronize(r.b));
    float t = 0;
    REG_CUDA(cudaEventElapsedTime(&t, r.a, r.b));
    ms[r.kind] += t;
    bytes[r.kind] += r.bytes;
    last_flops[r.kind] += r.flops;
    count[r.kind] += 1;
    pool.push_back(r.a);
    pool.push_back(r.b);
  }
  recs.clear();
}

ProfScope::ProfScope(int k, cudaStream_t st, double b, double f) : kind(k), s(st), bytes(b), flops(f) {
  if (tl_prof && (tl_prof->mask & (1u << k))) {
    a = tl_prof->take();
    REG_CUDA(cudaEventRecord(a, s));
  }
}

ProfScope::~ProfScope() {
  if (!a || !tl_prof) return;
  cudaEvent_t b = tl_prof->take();
  if (cudaEventRecord(b, s) != cudaSuccess) return;
  tl_prof->recs.push_back(KernelProfiler::Rec{kind, a, b, bytes, flops});
}

}  // namespace reg
