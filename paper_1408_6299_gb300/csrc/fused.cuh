// fused.cuh -- fused transport stages of the Heun sweeps (Mang & Biros,
// Eq. first-order-forward / first-order-adjoint / gauss-newton, Sec. 3.3.1).
//
// The stages work in a mixed domain: only the contiguous last axis is
// transformed to Fourier space (packed real-to-complex rows, see spectral.cu);
// a spectral derivative along any other axis a is applied to those rows as
// one column pass that runs the forward FFT along a, multiplies by i k~_a / n_a
// and runs the inverse FFT, all in shared memory. Then
//   d/dx_last u = C2R(i k_last R2C(u)),  d/dx_a u = C2R(D_a R2C(u)),
//   div q = C2R(i k_last Q_last + sum_a D_a Q_a),  Q_i = R2C(q_i).
// The last pass of a stage transforms all needed rows back to real space in
// one kernel and applies the stage's pointwise epilogue there:
//   advection  k = -v . grad u [- grad m . v~],  Heun update, optional store of grad u
//   divergence k = div(v lam),                   Heun update
// so a 3D stage costs four passes over the field and no separate pointwise
// kernel, and the gradient fields are never written unless they are kept.
#pragma once
#include <cuda.h>

#include "internal.h"

namespace reg {
namespace fused {

constexpr int kThreads = 256;

__host__ __device__ inline long kmask_l(long j, long n) { return j == n / 2 ? 0 : (j < n / 2 ? j : j - n); }
// the same for an index m < L held exactly in T (no integer conversion per element)
template <typename T, int L>
__device__ __forceinline__ T kmask_f(T m) {
  return m < (T)(L / 2) ? m : (m == (T)(L / 2) ? (T)0 : m - (T)L);
}

template <typename T, int NF>
struct RowsIn {
  const T* p[NF];
};
template <typename T, int NF>
struct RowsOut {
  cx<T>* p[NF];
};

// Packing step of the real-to-complex rows: buf holds, for NF x RB rows, the
// forward FFT of length M = L/2 of each row read as M complex values
// (x_{2j} + i x_{2j+1}); it writes the packed half spectrum of every row
// (slot 0 carries the DC and Nyquist values as re and im) to out[f]. Fields
// whose bit is set in zmask leave multiplied by i k_last (slot 0 -> 0).
template <typename T, int L, int RB, int NF>
__device__ __forceinline__ void r2c_pack(const cx<T>* buf, long row0, long nrows, cx<T>* const* out, int zmask,
                                         const cx<T>* __restrict__ twrc) {
  using C = cx<T>;
  constexpr int M = L / 2;
  constexpr int RS = padded_len(M);
  // M/2 work items per sequence (a power of two, so the item index splits by
  // shifts): item k >= 1 writes the modes k and M - k, item 0 the packed
  // DC/Nyquist slot and the middle mode M/2
  constexpr int Q2 = M / 2;
  for (int e = threadIdx.x; e < NF * RB * Q2; e += kThreads) {
    const int seq = e / Q2, item = e % Q2;
    const int f = seq / RB, r = seq % RB;
    const long row = row0 + r;
    if (row >= nrows) continue;
    C* o = out[f] + row * M;
    const C* b = buf + seq * RS;
    const bool dz = (zmask >> f) & 1;
    auto pair = [&](int k) {
      C zk = b[pad16(k)], zm = b[pad16(M - k)];
      C E = cscale(cadd(zk, cconj(zm)), (T)0.5);
      C Od = cscale(cmul_mi(csub(zk, cconj(zm))), (T)0.5);
      C t = cmul(__ldg(&twrc[k]), Od);
      C xk = cadd(E, t);
      C xm = cconj(csub(E, t));
      if (dz) {  // times i k
        xk = mk<C>(-(T)k * xk.y, (T)k * xk.x);
        xm = mk<C>(-(T)(M - k) * xm.y, (T)(M - k) * xm.x);
      }
      o[k] = xk;
      if (k != M - k) o[M - k] = xm;
    };
    if (item == 0) {
      C z0 = b[0];
      o[0] = dz ? mk<C>(0, 0) : mk<C>(z0.x + z0.y, z0.x - z0.y);
      pair(M / 2);
    } else {
      pair(item);
    }
  }
}

// Real-to-complex rows of NF fields in one block. PROD: field f is a_f * lam
// (pointwise), else in_f. Fields whose bit is set in zmask leave multiplied by
// i k_last (first derivative along the last axis; slot 0 -> 0).
template <typename T, int L, int RB, int NF, bool PROD>
__global__ void __launch_bounds__(kThreads) k_rows_r2c_n(RowsIn<T, NF> in, const T* __restrict__ lam,
                                                          RowsOut<T, NF> out, int zmask, long nrows,
                                                          const cx<T>* __restrict__ tw,
                                                          const cx<T>* __restrict__ twrc) {
  using C = cx<T>;
  constexpr int M = L / 2;
  constexpr int RS = padded_len(M);
  __shared__ C buf[NF * RB * RS];
  const long row0 = (long)blockIdx.x * RB;
  // all global loads of a thread are issued before the first shared store;
  // a thread takes every field of its points, so lam is read once per point
  constexpr int PER = (RB * M + kThreads - 1) / kThreads;
  C v[PER][NF];
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    int e = threadIdx.x + i * kThreads;
    long row = row0 + e / M;
    bool ok = e < RB * M && row < nrows;
    long q = row * M + e % M;
    C l = mk<C>(1, 1);
    if (PROD && ok) l = reinterpret_cast<const C*>(lam)[q];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      C z = ok ? reinterpret_cast<const C*>(in.p[f])[q] : mk<C>(0, 0);
      v[i][f] = PROD ? mk<C>(z.x * l.x, z.y * l.y) : z;
    }
  }
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    int e = threadIdx.x + i * kThreads;
    if (e < RB * M) {
#pragma unroll
      for (int f = 0; f < NF; ++f) buf[(f * RB + e / M) * RS + pad16(e % M)] = v[i][f];
    }
  }
  __syncthreads();
  smem_fft<T, M, false, kThreads, NF * RB>(buf, RS, tw);
  r2c_pack<T, L, RB, NF>(buf, row0, nrows, out.p, zmask, twrc);
}

// Epilogue parameters of the advection stage (state / incremental state).
template <typename T>
struct AdvEpi {
  const T* a[3];   // velocity components at the stage time
  const T* gm[3];  // source: grad m at the stage time (null: no source)
  const T* w[3];   // source: incremental velocity at the stage time
  const T* y;      // stage 1: y_j (null = 0); stage 2: acc
  T* out1;         // stage 1: y_j + h k; stage 2: acc + h/2 k (null: only keep grad u)
  T* out2;         // stage 1: y_j + h/2 k
  T* G[3];         // optional: keep grad u (null: not stored)
  const T* src;    // optional precomputed source sum_i gm_i w_i (used instead of gm/w)
  const T* sw[3];  // optional: with Sout, store Sout = sum_i (grad u)_i sw_i
  T* Sout;
  T h;
  int stage;
  int src_from_a;  // two-field stage, second field: the source is the first field's Sout value
  int a_from_a;    // two-field stage, second field: same velocity as the first (reuse its loaded values)
  int out1_spectral_only;  // out1 is only passed on as a spectrum (the row pass emits it): no real store
};

// Epilogue parameters of the divergence stage (adjoint / incremental adjoint).
// Stage 1 can also accumulate the body force f_l,i += cA_l y gmA_i (+ cB_l out1
// gmB_i): the trapezoid term of node j+1, or the two stage terms of the
// discrete adjoint. The accumulator is f_hi (+ f_lo) with layout [n_c][d][N];
// with f_lo set, (f_hi, f_lo) is a compensated pair (exact two-sum per add).
// Stage 0 only evaluates: out1 = div(v lam) (+ src). src (optional) is added
// to the divergence (the div(v~ lam) source of the full Newton incremental
// adjoint). gmC/yC (optional) add the Newton force term cA_l yC gmC_i.
template <typename T>
struct DivEpi {
  const T* y;  // stage 1: lam_{j+1}; stage 2: acc
  T* out1;
  T* out2;
  T h;
  int stage;
  T* f_hi;          // null: no force accumulation
  T* f_lo;          // null: plain accumulation into f_hi
  const T* gmA;     // d fields at stride N
  const T* gmB;     // d fields or null
  T cA[16], cB[16]; // per-coefficient weights
  int nc, d;
  long N;
  const T* src;     // added to the divergence
  const T* gmC;     // d fields or null
  const T* yC;
};

// The spectrum a one-field advection stage's complex-to-real pass emits for
// the next stage, so that stage needs no real-to-complex pass: the forward
// row transform of the stage's out1 values. out[0] receives the packed half
// spectrum of the rows the block itself read (row-local, so it may overwrite
// the pass's own input spectrum).
template <typename T>
struct Emit {
  cx<T>* out[1];
};

template <typename T, int NF>
struct RowsSpec {
  const cx<T>* p[NF];
};

// ADV2: two advection epilogues on 2 x d fields; DIVS: the divergence epilogue on
// the sum of the NF input spectra (added on load, one inverse transform)
enum { EPI_ADV = 1, EPI_DIV = 2, EPI_ADV2 = 3, EPI_DIVS = 4 };

// Hint: fetch a contiguous byte range into L2 (bulk prefetch; no completion to wait for).
__device__ __forceinline__ void l2_prefetch(const void* p, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(p), "r"(bytes) : "memory");
}

// The epilogue operands of one row block (elements [off, off + bytes) of each
// operand field) are requested into L2 while the block loads and transforms
// its spectra, so the epilogue finds them on chip. Threads 0..63 take one
// operand each; only operands the epilogue will read are requested.
template <typename T, int NF, int EPI>
__device__ __forceinline__ void prefetch_epilogue(const AdvEpi<T>& adv, const DivEpi<T>& dv, long off,
                                                  unsigned bytes, int first_thread = 0) {
  const int k = (int)threadIdx.x - first_thread;
  if (k < 0 || k >= 64) return;
  const T* p = nullptr;
  if (EPI == EPI_ADV) {
    if (adv.out1) {
      if (k < NF) p = adv.a[k];
      else if (k == NF) p = adv.y;
      else if (k == NF + 1) p = adv.src;
      else if (!adv.src && k < 2 * NF + 2) p = adv.gm[k - NF - 2];
      else if (!adv.src && adv.gm[0] && k < 3 * NF + 2) p = adv.w[k - 2 * NF - 2];
    }
    if (adv.Sout && k >= 32 && k < 32 + NF) p = adv.sw[k - 32];
  } else {
    const long N = dv.N;
    if (k == 0 && dv.stage >= 1) p = dv.y;
    else if (k == 1) p = dv.src;
    else if (dv.stage == 1 && dv.f_hi) {
      const int nf = dv.nc * dv.d;
      if (k == 2) p = dv.gmC ? dv.yC : nullptr;
      else if (k >= 3 && k < 3 + dv.d) p = dv.gmA + (k - 3) * N;
      else if (k >= 6 && k < 6 + dv.d) p = dv.gmB ? dv.gmB + (k - 6) * N : nullptr;
      else if (k >= 9 && k < 9 + dv.d) p = dv.gmC ? dv.gmC + (k - 9) * N : nullptr;
      else if (k >= 12 && k < 12 + nf) p = dv.f_hi + (long)(k - 12) * N;
      else if (k >= 12 + nf && k < 12 + 2 * nf) p = dv.f_lo ? dv.f_lo + (long)(k - 12 - nf) * N : nullptr;
    }
  }
  // the bulk prefetch wants a 16-byte aligned start (caller arrays may be offset views)
  if (p && ((reinterpret_cast<unsigned long long>(p + off) | bytes) & 15) == 0) l2_prefetch(p + off, bytes);
}

// Advection epilogue on the point pair q with the gradient components g[0..D)
// (-a.g [- source], Heun update, optional keep of g or of g.sw). srcv, when
// given, is the source value instead of e.src. Returns the Sout value.
// av_in: the velocity values at q (null: load them); av_out: receives the
// loaded velocity values when the Heun update ran.
template <typename T, int D>
__device__ __forceinline__ cx<T> adv_point(const AdvEpi<T>& e, const cx<T>* g, long q, const cx<T>* srcv,
                                           cx<T>* o1 = nullptr, const cx<T>* av_in = nullptr,
                                           cx<T>* av_out = nullptr) {
  using C = cx<T>;
  C so = mk<C>(0, 0);
  if (e.G[0]) {
#pragma unroll
    for (int f = 0; f < D; ++f) reinterpret_cast<C*>(e.G[f])[q] = g[f];
  }
  if (e.Sout) {
    T s0 = 0, s1 = 0;
#pragma unroll
    for (int f = 0; f < D; ++f) {
      C w = reinterpret_cast<const C*>(e.sw[f])[q];
      s0 += g[f].x * w.x;
      s1 += g[f].y * w.y;
    }
    so = mk<C>(s0, s1);
    reinterpret_cast<C*>(e.Sout)[q] = so;
  }
  if (!e.out1) return so;
  T k0 = 0, k1 = 0;
#pragma unroll
  for (int f = 0; f < D; ++f) {
    C a = av_in ? av_in[f] : reinterpret_cast<const C*>(e.a[f])[q];
    if (av_out) av_out[f] = a;
    k0 -= a.x * g[f].x;
    k1 -= a.y * g[f].y;
  }
  if (srcv) {
    k0 -= srcv->x;
    k1 -= srcv->y;
  } else if (e.src) {
    C sv = reinterpret_cast<const C*>(e.src)[q];
    k0 -= sv.x;
    k1 -= sv.y;
  } else if (e.gm[0]) {
#pragma unroll
    for (int f = 0; f < D; ++f) {
      C gm = reinterpret_cast<const C*>(e.gm[f])[q];
      C w = reinterpret_cast<const C*>(e.w[f])[q];
      k0 -= gm.x * w.x;
      k1 -= gm.y * w.y;
    }
  }
  C r1;
  if (e.stage == 1) {
    C yv = e.y ? reinterpret_cast<const C*>(e.y)[q] : mk<C>(0, 0);
    r1 = mk<C>(yv.x + e.h * k0, yv.y + e.h * k1);
    reinterpret_cast<C*>(e.out2)[q] = mk<C>(yv.x + (T)0.5 * e.h * k0, yv.y + (T)0.5 * e.h * k1);
  } else {
    C yv = reinterpret_cast<const C*>(e.y)[q];
    r1 = mk<C>(yv.x + (T)0.5 * e.h * k0, yv.y + (T)0.5 * e.h * k1);
  }
  if (!e.out1_spectral_only) reinterpret_cast<C*>(e.out1)[q] = r1;
  if (o1) *o1 = r1;
  return so;
}

// Divergence epilogue on the point pair q with the divergence value k (scaled,
// real space): Heun stage update and, in stage 1, the optional body-force
// accumulation (see DivEpi).
template <typename T>
__device__ __forceinline__ void div_point(const DivEpi<T>& dv, cx<T> k, long q) {
  using C = cx<T>;
  if (dv.src) {
    C sv = reinterpret_cast<const C*>(dv.src)[q];
    k = mk<C>(k.x + sv.x, k.y + sv.y);
  }
  if (dv.stage == 0) {
    reinterpret_cast<C*>(dv.out1)[q] = k;
    return;
  }
  C yv = reinterpret_cast<const C*>(dv.y)[q];
  if (dv.stage != 1) {
    reinterpret_cast<C*>(dv.out1)[q] = mk<C>(yv.x + (T)0.5 * dv.h * k.x, yv.y + (T)0.5 * dv.h * k.y);
    return;
  }
  C o1 = mk<C>(yv.x + dv.h * k.x, yv.y + dv.h * k.y);
  reinterpret_cast<C*>(dv.out1)[q] = o1;
  reinterpret_cast<C*>(dv.out2)[q] = mk<C>(yv.x + (T)0.5 * dv.h * k.x, yv.y + (T)0.5 * dv.h * k.y);
  if (!dv.f_hi) return;
  // products of the point pair with every component, then per coefficient
  // all loads before any store
  C ta[3], tb[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    ta[i] = tb[i] = mk<C>(0, 0);
    if (i < dv.d) {
      C ga = reinterpret_cast<const C*>(dv.gmA + i * dv.N)[q];
      ta[i] = mk<C>(yv.x * ga.x, yv.y * ga.y);
      if (dv.gmC) {
        C gc = reinterpret_cast<const C*>(dv.gmC + i * dv.N)[q];
        C yc = reinterpret_cast<const C*>(dv.yC)[q];
        ta[i] = mk<C>(ta[i].x + yc.x * gc.x, ta[i].y + yc.y * gc.y);
      }
      if (dv.gmB) {
        C gb = reinterpret_cast<const C*>(dv.gmB + i * dv.N)[q];
        tb[i] = mk<C>(o1.x * gb.x, o1.y * gb.y);
      }
    }
  }
  for (int l = 0; l < dv.nc; ++l) {
    C hi[3], lo[3];
    C* Hf = reinterpret_cast<C*>(dv.f_hi + (long)l * dv.d * dv.N);
    C* Lo = dv.f_lo ? reinterpret_cast<C*>(dv.f_lo + (long)l * dv.d * dv.N) : nullptr;
    const long hN = dv.N / 2;
#pragma unroll
    for (int i = 0; i < 3; ++i)
      if (i < dv.d) {
        hi[i] = Hf[i * hN + q];
        lo[i] = Lo ? Lo[i * hN + q] : mk<C>(0, 0);
      }
#pragma unroll
    for (int i = 0; i < 3; ++i)
      if (i < dv.d) {
        T t0 = dv.cA[l] * ta[i].x + dv.cB[l] * tb[i].x;
        T t1 = dv.cA[l] * ta[i].y + dv.cB[l] * tb[i].y;
        if (Lo) {
          C h = hi[i];
          T s0 = h.x + t0, b0 = s0 - h.x, s1 = h.y + t1, b1 = s1 - h.y;
          lo[i].x += (h.x - (s0 - b0)) + (t0 - b0);
          lo[i].y += (h.y - (s1 - b1)) + (t1 - b1);
          Hf[i * hN + q] = mk<C>(s0, s1);
          Lo[i * hN + q] = lo[i];
        } else {
          Hf[i * hN + q] = mk<C>(hi[i].x + t0, hi[i].y + t1);
        }
      }
  }
}

// ---------------------------------------------------------------------------
// Edge stage of the two-stage forward row transforms (Plan<M>: M = R0 * R1).
// The last stage runs in registers and feeds the pack directly: butterfly
// j < R0 of a sequence yields the modes k = j + R0 r (r < R1). The pack
// combines mode k with mode M - k, which sits in butterfly (R0 - j) mod R0 at
// r' = R1 - 1 - r (for j = 0 in the same butterfly at (R1 - r) mod R1). The
// R0 butterflies of a sequence are neighbouring lanes of one warp, so the
// partner values arrive by warp shuffles instead of a shared-memory round
// trip, and each lane packs only its own modes.
// ---------------------------------------------------------------------------
template <int M>
struct Edge {
  static constexpr int R0 = Plan<M>::R[0], R1 = Plan<M>::R[1];
  // two stages, at most 8 values per edge butterfly (a lane holds them and
  // its partner's), whole sequences inside a warp: M = 32, 64, 128
  static constexpr bool ok = Plan<M>::S == 2 && R1 <= 8 && R0 <= 32 && 32 % R0 == 0;
};

// p[r] = value of mode M - k for k = j + R0 r, given this lane's x[r] (mode k).
// Every lane of the warp must call it (full-warp shuffles).
template <typename T, int R0, int R1>
__device__ __forceinline__ void edge_partners(const cx<T> (&x)[R1], cx<T> (&p)[R1], int j) {
  const int lane = threadIdx.x & 31;
  const int src = lane - j + ((R0 - j) & (R0 - 1));
#pragma unroll
  for (int r = 0; r < R1; ++r) {
    const cx<T> v = x[R1 - 1 - r];
    const T a = __shfl_sync(0xffffffffu, v.x, src);
    const T b = __shfl_sync(0xffffffffu, v.y, src);
    p[r] = j == 0 ? x[(R1 - r) % R1] : mk<cx<T>>(a, b);
  }
}

// Forward pack of mode k >= 1 of a real row from the complex FFT values zk =
// Z[k], zm = Z[M - k] of its M complex pairs: X[k] = E + W^k Od with E =
// (zk + conj zm)/2, Od = -i (zk - conj zm)/2. dz: times i k (last-axis derivative).
template <typename T>
__device__ __forceinline__ cx<T> pack_mode(int k, cx<T> zk, cx<T> zm, const cx<T>* __restrict__ twrc, bool dz) {
  using C = cx<T>;
  C E = cscale(cadd(zk, cconj(zm)), (T)0.5);
  C Od = cscale(cmul_mi(csub(zk, cconj(zm))), (T)0.5);
  C xk = cadd(E, cmul(__ldg(&twrc[k]), Od));
  if (dz) xk = mk<C>(-(T)k * xk.y, (T)k * xk.x);
  return xk;
}
// the packed slot 0 (DC + i Nyquist) from Z[0]
template <typename T>
__device__ __forceinline__ cx<T> pack_slot0(cx<T> z0, bool dz) {
  return dz ? mk<cx<T>>(0, 0) : mk<cx<T>>(z0.x + z0.y, z0.x - z0.y);
}
// Edge stage of the forward row transforms and the pack: S sequences of RS
// padded values in buf after the first stage (radix R0, Stockham order);
// sequence s is field s / RB, row row0 + s % RB, written to out[s / RB].
// All NT threads call it.
template <typename T, int M, int RB, int S, int NT>
__device__ __forceinline__ void edge_forward_pack(const cx<T>* buf, long row0, long nrows, cx<T>* const* out,
                                                  int zmask, const cx<T>* __restrict__ tw1,
                                                  const cx<T>* __restrict__ twrc) {
  constexpr int NO = S / RB;  // output fields
  using C = cx<T>;
  constexpr int R0 = Edge<M>::R0, R1 = Edge<M>::R1, RS = padded_len(M);
  constexpr int TASKS = S * R0;
  static_assert(NT % 32 == 0, "whole warps");
#pragma unroll
  for (int it = 0; it < (TASKS + NT - 1) / NT; ++it) {
    const int u = threadIdx.x + it * NT;
    if (u - (int)(threadIdx.x & 31) >= TASKS) break;  // the whole warp is past the end (uniform)
    const bool act = u < TASKS;
    const int seq = act ? u / R0 : 0, j = u % R0;
    const C* b = buf + seq * RS;
    C x[R1];
#pragma unroll
    for (int r = 0; r < R1; ++r) x[r] = b[pad16(j + R0 * r)];
#pragma unroll
    for (int r = 1; r < R1; ++r) x[r] = cmul(x[r], __ldg(&tw1[r * R0 + j]));
    Dft<T, R1>::run(x);
    C p[R1];
    edge_partners<T, R0, R1>(x, p, j);
    const long row = row0 + seq % RB;
    if (act && row < nrows) {
      const int f = seq / RB;
      const bool dz = (zmask >> f) & 1;
      C* o = out[0];  // the field's pointer by selection (constant indices only)
#pragma unroll
      for (int g = 1; g < NO; ++g)
        if (f == g) o = out[g];
      o += row * M;
#pragma unroll
      for (int r = 0; r < R1; ++r) {
        const int k = j + R0 * r;
        o[k] = (r == 0 && j == 0) ? pack_slot0<T>(x[0], dz) : pack_mode<T>(k, x[r], p[r], twrc, dz);
      }
    }
  }
}

// Stage epilogue of rows row0..row0+RB-1 from the inverse transforms in buf
// (NF sequences x RB rows of RS padded values, natural order, conjugated and
// unscaled), each thread taking the point pairs threadIdx.x + it * NT.
// NE = 1 (advection only): the block then transforms the epilogue's out1
// values forward in the same buffer and writes their packed spectrum to
// em.out[0].
template <typename T, int L, int RB, int NF, int EPI, int NE, int NT>
__device__ __forceinline__ void c2r_tail(cx<T>* buf, long row0, long nrows, const AdvEpi<T>& adv,
                                         const DivEpi<T>& dv, const cx<T>* __restrict__ tw,
                                         const cx<T>* __restrict__ twrc, const AdvEpi<T>& advB,
                                         const Emit<T>& em) {
  using C = cx<T>;
  static_assert(NE == 0 || (NE == 1 && EPI == EPI_ADV), "only one-field advection stages emit a spectrum");
  constexpr int M = L / 2;
  constexpr int RS = padded_len(M);
  const T s = (T)1 / (T)M;
  constexpr int ITER = (RB * M + NT - 1) / NT;
  constexpr int NEA = NE > 0 ? NE : 1;
  C ev[ITER][NEA];  // emitted values (point pairs) of this thread
#pragma unroll
  for (int it = 0; it < ITER; ++it) {
    const int e = threadIdx.x + it * NT;
#pragma unroll
    for (int f = 0; f < NEA; ++f) ev[it][f] = mk<C>(0, 0);
    if (e >= RB * M) continue;
    int r = e / M, j = e % M;
    long row = row0 + r;
    if (row >= nrows) continue;
    const long q = row * M + j;  // index of the point pair (2j, 2j+1) of this row
    C g[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      C z = buf[(f * RB + r) * RS + pad16(j)];
      g[f] = mk<C>(z.x * s, -z.y * s);
    }
    if (EPI == EPI_ADV) {
      adv_point<T, NF>(adv, g, q, nullptr, &ev[it][0]);
    } else if (EPI == EPI_ADV2) {
      C av[NF / 2 > 0 ? NF / 2 : 1];
      const C sa = adv_point<T, NF / 2>(adv, g, q, nullptr, nullptr, nullptr, av);
      adv_point<T, NF / 2>(advB, g + NF / 2, q, advB.src_from_a ? &sa : nullptr, nullptr,
                           advB.a_from_a ? av : nullptr);
    } else {
      div_point<T>(dv, g[0], q);
    }
  }
  if constexpr (NE > 0) {
    // the forward row transform of the emitted values, as the r2c pass does it
    __syncthreads();  // every thread has read the inverse transforms from buf
#pragma unroll
    for (int it = 0; it < ITER; ++it) {
      const int e = threadIdx.x + it * NT;
      if (e < RB * M) {
#pragma unroll
        for (int f = 0; f < NE; ++f) buf[(f * RB + e / M) * RS + pad16(e % M)] = ev[it][f];
      }
    }
    __syncthreads();
    if constexpr (sizeof(T) == 4 && Edge<M>::ok) {
      stockham_stage<T, M, Edge<M>::R0, 1, false, NT, NE * RB>(buf, RS, tw);
      edge_forward_pack<T, M, RB, NE * RB, NT>(buf, row0, nrows, em.out, 0, tw + stage_tw_offset(M, 1), twrc);
    } else {
      smem_fft<T, M, false, NT, NE * RB>(buf, RS, tw);
      r2c_pack<T, L, RB, NE>(buf, row0, nrows, em.out, 0, twrc);
    }
  }
}

// Inverse row transforms of one staged row block (NF fields x RB rows in buf,
// padded rows of RS, already unpacked from the half spectra and conjugated),
// then the stage epilogue. Called by all threads of the block after buf is complete.
template <typename T, int L, int RB, int NF, int EPI, int NE>
__device__ __forceinline__ void c2r_block(cx<T>* buf, long row0, long nrows, const AdvEpi<T>& adv,
                                          const DivEpi<T>& dv, const cx<T>* __restrict__ tw,
                                          const cx<T>* __restrict__ twrc, const AdvEpi<T>& advB,
                                          const Emit<T>& em) {
  smem_fft<T, L / 2, false, kThreads, NF * RB>(buf, padded_len(L / 2), tw);
  c2r_tail<T, L, RB, NF, EPI, NE, kThreads>(buf, row0, nrows, adv, dv, tw, twrc, advB, em);
}


// Complex-to-real rows of NF fields, then the stage epilogue on the real
// values (each thread handles a pair of neighbouring points). Fields whose
// bit is set in zmask are multiplied by i k_last on load.
template <typename T, int L, int RB, int NF, int EPI, int NE>
// single precision: at most 40 registers, six resident blocks per SM. Measured on the 256^3 matvec:
// 285.0 -> 280.5 ms against five; the divergence epilogue spills a few words and still gains. The
// variant that also emits the next stage's spectrum runs five blocks (measured better than six,
// four and three).
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? (NE > 0 ? 5 : 6) : 1) k_rows_c2r_n(RowsSpec<T, NF> in, int zmask, AdvEpi<T> adv,
                                                          DivEpi<T> dv, long nrows, const cx<T>* __restrict__ tw,
                                                          const cx<T>* __restrict__ twrc, AdvEpi<T> advB,
                                                          Emit<T> em) {
  using C = cx<T>;
  constexpr int M = L / 2;
  constexpr int RS = padded_len(M);
  constexpr int NX = EPI == EPI_DIVS ? 1 : NF;  // sequences transformed per row
  constexpr int NB = NX > NE ? NX : NE;         // sequences the buffer holds
  __shared__ C buf[NB * RB * RS];
  const long row0 = (long)blockIdx.x * RB;
  // Prologue: M/2 work items per sequence; item k >= 1 loads the modes k and
  // M - k of its row, item 0 the packed DC/Nyquist slot and the middle mode
  // M/2. Each applies the z-derivative (zmask; the DIVS form adds its inputs)
  // and unpacks the half spectrum for the complex inverse transform in
  // registers, so buf is filled by one store pass.
  constexpr int Q2 = M / 2;
  constexpr int PER = (NX * RB * Q2 + kThreads - 1) / kThreads;
  C va[PER], vb[PER];
  auto mode = [&](int f, long row, int k) {
    C z = mk<C>(0, 0);
    if constexpr (EPI == EPI_DIVS) {
#pragma unroll
      for (int g = 0; g < NF; ++g) {
        C x = in.p[g][row * M + k];
        if ((zmask >> g) & 1) x = mk<C>(-(T)k * x.y, (T)k * x.x);
        z = cadd(z, x);
      }
    } else {
      z = in.p[f][row * M + k];
      if ((zmask >> f) & 1) z = mk<C>(-(T)k * z.y, (T)k * z.x);
    }
    return z;
  };
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int e = threadIdx.x + i * kThreads;
    va[i] = vb[i] = mk<C>(0, 0);
    if (e < NX * RB * Q2) {
      const int seq = e / Q2, item = e % Q2;
      const long row = row0 + seq % RB;
      if (row < nrows) {
        va[i] = mode(seq / RB, row, item);
        vb[i] = mode(seq / RB, row, item == 0 ? M / 2 : M - item);
      }
    }
  }
  // operand slices of at most 8 KB: larger blocks would prefetch more than the
  // resident blocks of the whole GPU keep in L2 (measured: re-read traffic)
  if constexpr (RB * L * sizeof(T) <= 8192) {
    const long nr = nrows - row0 < RB ? nrows - row0 : RB;
    if constexpr (EPI == EPI_ADV2) {
      prefetch_epilogue<T, NF / 2, EPI_ADV>(adv, dv, row0 * L, (unsigned)(nr * L * sizeof(T)));
      prefetch_epilogue<T, NF / 2, EPI_ADV>(advB, dv, row0 * L, (unsigned)(nr * L * sizeof(T)), 64);
    } else {
      prefetch_epilogue<T, NF, EPI>(adv, dv, row0 * L, (unsigned)(nr * L * sizeof(T)));
    }
  }
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int e = threadIdx.x + i * kThreads;
    if (e < NX * RB * Q2) {
      const int seq = e / Q2, item = e % Q2;
      C* b = buf + seq * RS;
      // modes k and M - k of the half spectrum -> complex sequence values (conjugated:
      // the inverse runs as a forward FFT)
      auto unpack = [&](int k, C xk, C xm) {
        C E = cscale(cadd(xk, cconj(xm)), (T)0.5);
        C Od = cscale(cmul(csub(xk, cconj(xm)), cconj(__ldg(&twrc[k]))), (T)0.5);
        C zk = mk<C>(E.x - Od.y, E.y + Od.x);
        C zm = mk<C>(E.x + Od.y, -E.y + Od.x);
        b[pad16(k)] = cconj(zk);
        if (k != M - k) b[pad16(M - k)] = cconj(zm);
      };
      if (item == 0) {
        const C p = va[i];
        b[0] = cconj(mk<C>((p.x + p.y) * (T)0.5, (p.x - p.y) * (T)0.5));
        unpack(M / 2, vb[i], vb[i]);
      } else {
        unpack(item, va[i], vb[i]);
      }
    }
  }
  __syncthreads();
  c2r_block<T, L, RB, NX, EPI, NE>(buf, row0, nrows, adv, dv, tw, twrc, advB, em);
}

// ---------------------------------------------------------------------------
// Real-to-complex row pass on the edge-stage transforms (Edge<M>::ok): the
// first stage (radix R0) straight from global memory, then the edge stage
// plus pack in registers, so the block's values cross shared memory once.
// The complex-to-real counterpart is k_rows_c2r_p (after the copy helpers).
// ---------------------------------------------------------------------------
template <typename T, int L, int RB, int NF, bool PROD, int NT>
__global__ void __launch_bounds__(NT) k_rows_r2c_e(RowsIn<T, NF> in, const T* __restrict__ lam,
                                                    RowsOut<T, NF> out, int zmask, long nrows,
                                                    const cx<T>* __restrict__ tw, const cx<T>* __restrict__ twrc) {
  using C = cx<T>;
  constexpr int M = L / 2, R0 = Edge<M>::R0, R1 = Edge<M>::R1, RS = padded_len(M);
  static_assert(Edge<M>::ok, "edge-stage plan");
  __shared__ C buf[NF * RB * RS];
  const long row0 = (long)blockIdx.x * RB;
  // first stage: butterfly j < R1 of a sequence takes the complex pairs j + R1 r (r < R0)
  constexpr int T0 = NF * RB * R1;
#pragma unroll
  for (int it = 0; it < (T0 + NT - 1) / NT; ++it) {
    const int u = threadIdx.x + it * NT;
    if (u < T0) {
      const int seq = u / R1, j = u % R1;
      const long row = row0 + seq % RB;
      C v[R0];
      if (row < nrows) {
        const long q = row * M + j;
        const T* src = in.p[0];
#pragma unroll
        for (int g = 1; g < NF; ++g)
          if (seq / RB == g) src = in.p[g];
        const C* x = reinterpret_cast<const C*>(src) + q;
#pragma unroll
        for (int r = 0; r < R0; ++r) {
          C z = x[r * R1];
          if (PROD) {
            const C l = reinterpret_cast<const C*>(lam)[q + r * R1];
            z = mk<C>(z.x * l.x, z.y * l.y);
          }
          v[r] = z;
        }
      } else {
#pragma unroll
        for (int r = 0; r < R0; ++r) v[r] = mk<C>(0, 0);
      }
      Dft<T, R0>::run(v);
      C* b = buf + seq * RS;
#pragma unroll
      for (int r = 0; r < R0; ++r) b[pad16(j * R0 + r)] = v[r];
    }
  }
  __syncthreads();
  edge_forward_pack<T, M, RB, NF * RB, NT>(buf, row0, nrows, out.p, zmask, tw + stage_tw_offset(M, 1), twrc);
}

// Spectral derivative along a strided axis of length L on z-spectral rows:
// out = IFFT_a(i k~_a FFT_a(in)) (+ add). Element j of pencil (outer, inner)
// at offset outer*L*s + j*s + inner; a block takes TC neighbouring inners.
// in == out and add == out are allowed (each block reads its tile first).
template <typename T, int L, int TC>
__global__ void __launch_bounds__(kThreads) k_cols_deriv(const cx<T>* in, cx<T>* out, const cx<T>* add, long s,
                                                          const cx<T>* __restrict__ tw) {
  using C = cx<T>;
  __shared__ C buf[L * TC];
  const long off = (long)blockIdx.y * L * s + (long)blockIdx.x * TC;
  constexpr int PER = (L * TC + kThreads - 1) / kThreads;
  C v[PER];
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    int e = threadIdx.x + i * kThreads;
    if (e < L * TC) v[i] = in[off + (long)(e / TC) * s + (e % TC)];
  }
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    int e = threadIdx.x + i * kThreads;
    if (e < L * TC) buf[e] = v[i];
  }
  __syncthreads();
  smem_fft<T, L, true, kThreads, TC>(buf, TC, tw);
  const T sc = (T)1 / (T)L;
  for (int e = threadIdx.x; e < L * TC; e += kThreads) {
    int j = e / TC;
    T k = kmask_f<T, L>((T)j) * sc;
    C z = buf[e];
    buf[e] = cconj(mk<C>(-k * z.y, k * z.x));  // conjugated: the inverse runs as a forward FFT
  }
  __syncthreads();
  smem_fft<T, L, true, kThreads, TC>(buf, TC, tw);
  for (int e = threadIdx.x; e < L * TC; e += kThreads) {
    int j = e / TC, c = e % TC;
    C z = cconj(buf[e]);
    long o = off + (long)j * s + c;
    if (add) z = cadd(z, add[o]);
    out[o] = z;
  }
}

// Same operator for lengths with a two-stage radix plan L = R0*R1, kept in
// registers between stages. Forward: stage A (radix R0) straight from global
// memory, shared exchange, stage B (radix R1, twiddles W_L^{r j}). After stage
// B a thread holds the frequencies j + r*R0 (r < R1) of one column, which are
// exactly the inputs of the first stage of an inverse transform planned as
// (R1, R0); the multiplier and the conjugation happen in registers, then the
// inverse stage A' (radix R1), a shared exchange, and stage B' (radix R0,
// twiddles W_L^{r k} read transposed from the same table) writes to global
// memory. Thread t owns column t % TC.
template <typename T, int L, int TC, int R0, int R1>
__global__ void __launch_bounds__(TC * (R0 > L / R0 ? R0 : L / R0)) k_cols_deriv2(const cx<T>* in, cx<T>* out,
                                                                                    const cx<T>* add, long s,
                                                                                    const cx<T>* __restrict__ tw) {
  using C = cx<T>;
  constexpr int Q0 = L / R0;  // tasks per column of the radix-R0 stages
  constexpr int Q1 = R0;      // tasks per column of the radix-R1 stages (L / R1)
  __shared__ C buf[L * TC];
  const long off = (long)blockIdx.y * L * s + (long)blockIdx.x * TC;
  const int b = threadIdx.x % TC, j = threadIdx.x / TC;
  C v[R0 > R1 ? R0 : R1];
  // forward stage A: x[j + r*Q0], r < R0
  if (j < Q0) {
#pragma unroll
    for (int r = 0; r < R0; ++r) v[r] = in[off + (long)(j + r * Q0) * s + b];
    Dft<T, R0>::run(v);
#pragma unroll
    for (int r = 0; r < R0; ++r) buf[(j * R0 + r) * TC + b] = v[r];
  }
  __syncthreads();
  const T sc = (T)1 / (T)L;
  const T jf = (T)j;
  if (j < Q1) {
    // forward stage B: positions j + r*R0, twiddle W_L^{r j}
#pragma unroll
    for (int r = 0; r < R1; ++r) v[r] = buf[(j + r * R0) * TC + b];
#pragma unroll
    for (int r = 1; r < R1; ++r) v[r] = cmul(v[r], __ldg(&tw[r * R0 + j]));
    Dft<T, R1>::run(v);
    // v[r] is frequency j + r*R0: conj(i k~ z / L) = (-k z.y, -k z.x) with k = k~ / L
#pragma unroll
    for (int r = 0; r < R1; ++r) {
      T k = kmask_f<T, L>(jf + (T)(r * R0)) * sc;
      v[r] = mk<C>(-k * v[r].y, -k * v[r].x);
    }
    // inverse stage A' (radix R1) on the same values: inputs j + r*R0 = j + r*(L/R1)
    Dft<T, R1>::run(v);
  }
  __syncthreads();  // every thread has finished reading buf in stage B
  if (j < Q1) {
#pragma unroll
    for (int r = 0; r < R1; ++r) buf[(j * R1 + r) * TC + b] = v[r];
  }
  __syncthreads();
  if (j < Q0) {
    // inverse stage B' (radix R0, previous radices R1): positions j + r*R1,
    // twiddle W_L^{r j} = table entry [j*R0 + r]
#pragma unroll
    for (int r = 0; r < R0; ++r) v[r] = buf[(j + r * Q0) * TC + b];
#pragma unroll
    for (int r = 1; r < R0; ++r) v[r] = cmul(v[r], __ldg(&tw[j * R0 + r]));
    Dft<T, R0>::run(v);
#pragma unroll
    for (int r = 0; r < R0; ++r) {
      C z = cconj(v[r]);
      long o = off + (long)(j + r * Q0) * s + b;
      if (add) z = cadd(z, add[o]);
      out[o] = z;
    }
  }
}

// ---------------------------------------------------------------------------
// Persistent, double-buffered form of k_cols_deriv2: each block walks tiles
// t = blockIdx.x, blockIdx.x + gridDim.x, ...; while it transforms tile t in
// one shared buffer, asynchronous copies (cp.async, 16 bytes each) bring
// tile t + gridDim.x into the other, so the memory system keeps streaming
// during the FFT stages. A tile is TC neighbouring columns x L rows.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

template <typename T, int L, int TC, int NT>
__device__ __forceinline__ void tile_prefetch(cx<T>* dst, const cx<T>* in, long off, long s) {
  constexpr int PER16 = 16 / sizeof(cx<T>);  // complex values per 16-byte copy
  constexpr int CHUNKS = L * TC / PER16;
  for (int e = threadIdx.x; e < CHUNKS; e += NT) {
    int row = (e * PER16) / TC, col = (e * PER16) % TC;
    cp_async16(dst + row * TC + col, in + off + (long)row * s + col);
  }
}

template <typename T, int L, int TC, int R0, int R1>
__global__ void __launch_bounds__(TC * (R0 > L / R0 ? R0 : L / R0)) k_cols_deriv2p(const cx<T>* in, cx<T>* out,
                                                                                     const cx<T>* add, long s,
                                                                                     int ntx, int ntiles,
                                                                                     const cx<T>* __restrict__ tw) {
  using C = cx<T>;
  constexpr int Q0 = L / R0;
  constexpr int Q1 = R0;
  constexpr int NT = TC * (Q0 > Q1 ? Q0 : Q1);
  extern __shared__ __align__(128) unsigned char smem_raw[];
  C* bufs = reinterpret_cast<C*>(smem_raw);  // two tiles of L*TC
  const int b = threadIdx.x % TC, j = threadIdx.x / TC;
  const T sc = (T)1 / (T)L;
  const T jf = (T)j;
  C v[R0 > R1 ? R0 : R1];
  // tile t covers columns (t % ntx)*TC.. of pencil block t / ntx (32-bit division: the 64-bit
  // routine runs partly on the narrow FP64 pipe)
  auto tile_off = [&](int tt) { return (long)(tt / ntx) * L * s + (long)(tt % ntx) * TC; };
  int t = blockIdx.x;
  if (t < ntiles) tile_prefetch<T, L, TC, NT>(bufs, in, tile_off(t), s);
  cp_async_commit();
  for (int it = 0; t < ntiles; t += gridDim.x, ++it) {
    C* cur = bufs + (it & 1) * L * TC;
    C* nxt = bufs + ((it + 1) & 1) * L * TC;
    const long off = tile_off(t);
    const int tn = t + gridDim.x;
    if (tn < ntiles) tile_prefetch<T, L, TC, NT>(nxt, in, tile_off(tn), s);
    cp_async_commit();
    cp_async_wait_prev();  // this tile's copies have landed (the newest group may still fly)
    __syncthreads();
    // forward stage A from the staged tile
    if (j < Q0) {
#pragma unroll
      for (int r = 0; r < R0; ++r) v[r] = cur[(j + r * Q0) * TC + b];
      Dft<T, R0>::run(v);
    }
    __syncthreads();
    if (j < Q0) {
#pragma unroll
      for (int r = 0; r < R0; ++r) cur[(j * R0 + r) * TC + b] = v[r];
    }
    __syncthreads();
    if (j < Q1) {
#pragma unroll
      for (int r = 0; r < R1; ++r) v[r] = cur[(j + r * R0) * TC + b];
#pragma unroll
      for (int r = 1; r < R1; ++r) v[r] = cmul(v[r], __ldg(&tw[r * R0 + j]));
      Dft<T, R1>::run(v);
#pragma unroll
      for (int r = 0; r < R1; ++r) {
        T k = kmask_f<T, L>(jf + (T)(r * R0)) * sc;
        v[r] = mk<C>(-k * v[r].y, -k * v[r].x);
      }
      Dft<T, R1>::run(v);
    }
    __syncthreads();
    if (j < Q1) {
#pragma unroll
      for (int r = 0; r < R1; ++r) cur[(j * R1 + r) * TC + b] = v[r];
    }
    __syncthreads();
    if (j < Q0) {
#pragma unroll
      for (int r = 0; r < R0; ++r) v[r] = cur[(j + r * Q0) * TC + b];
#pragma unroll
      for (int r = 1; r < R0; ++r) v[r] = cmul(v[r], __ldg(&tw[j * R0 + r]));
      Dft<T, R0>::run(v);
#pragma unroll
      for (int r = 0; r < R0; ++r) {
        C z = cconj(v[r]);
        long o = off + (long)(j + r * Q0) * s + b;
        if (add) z = cadd(z, add[o]);
        out[o] = z;
      }
    }
    __syncthreads();  // cur is refilled by the prefetch of the iteration after next
  }
  cp_async_wait_prev();
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// ---------------------------------------------------------------------------
// TMA form of k_cols_deriv2p: one thread brings each tile (TC columns x L
// rows of the strided pencils) into shared memory with a 2D tensor copy
// (cp.async.bulk.tensor) that completes on an mbarrier; the other threads
// issue no copy instructions. Every wait is bounded: a block whose copy does
// not land within the bound counts a timeout in g_tma_timeouts (read by the
// host) and stops.
// ---------------------------------------------------------------------------
static __device__ int g_tma_timeouts;

__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
// wait for the phase with parity `parity`; false when the bound runs out
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, int tries = 1 << 20) {
  for (int i = 0; i < tries; ++i) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::
          "r"(smem_addr(dst)),
      "l"(map), "r"(x), "r"(y), "r"(smem_addr(bar))
      : "memory");
}

// Failure-path check: one block waits on an mbarrier that nothing completes,
// gives up after `tries` polls and counts the timeout as the column pass does.
static __global__ void k_wait_timeout_probe(int tries) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  if (!__syncthreads_and(mbar_wait(&bar, 0, tries)) && threadIdx.x == 0) atomicAdd(&g_tma_timeouts, 1);
}

// The tensor map views the input as rows of s complex values (4-byte
// elements, s * sizeof(cx<T>) / 4 per row) and outer * L rows; tile t is the
// box at x = (t % ntx) * TC complex values, y = (t / ntx) * L rows.
template <typename T, int L, int TC, int R0, int R1>
__global__ void __launch_bounds__(TC * (R0 > L / R0 ? R0 : L / R0)) k_cols_deriv2t(const __grid_constant__ CUtensorMap tmap,
                                                                                     cx<T>* out, const cx<T>* add, long s,
                                                                                     int ntx, int ntiles,
                                                                                     const cx<T>* __restrict__ tw) {
  using C = cx<T>;
  constexpr int Q0 = L / R0;
  constexpr int Q1 = R0;
  constexpr unsigned TILE_BYTES = L * TC * sizeof(C);
  constexpr int XW = TC * (int)sizeof(C) / 4;  // box width in 4-byte elements
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar[2];
  C* bufs = reinterpret_cast<C*>(smem_raw);  // two tiles of L*TC
  const int b = threadIdx.x % TC, j = threadIdx.x / TC;
  const T sc = (T)1 / (T)L;
  const T jf = (T)j;
  C v[R0 > R1 ? R0 : R1];
  auto tile_off = [&](int tt) { return (long)(tt / ntx) * L * s + (long)(tt % ntx) * TC; };
  auto issue = [&](int tt, int buf) {  // one thread
    mbar_expect_tx(&bar[buf], TILE_BYTES);
    tma_load_2d(bufs + buf * L * TC, &tmap, (tt % ntx) * XW, (tt / ntx) * L, &bar[buf]);
  };
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  int t = blockIdx.x;
  if (threadIdx.x == 0 && t < ntiles) issue(t, 0);
  int it = 0;
  bool pending_other = false;  // a copy into the other buffer is in flight
  for (; t < ntiles; t += gridDim.x, ++it) {
    const int cb = it & 1;
    C* cur = bufs + cb * L * TC;
    const long off = tile_off(t);
    const int tn = t + gridDim.x;
    pending_other = tn < ntiles;
    if (threadIdx.x == 0 && pending_other) issue(tn, cb ^ 1);
    // all threads agree on the outcome, so a timeout ends the whole block together
    if (!__syncthreads_and(mbar_wait(&bar[cb], (it >> 1) & 1))) {
      if (threadIdx.x == 0) atomicAdd(&g_tma_timeouts, 1);
      break;
    }
    // forward stage A from the staged tile
    if (j < Q0) {
#pragma unroll
      for (int r = 0; r < R0; ++r) v[r] = cur[(j + r * Q0) * TC + b];
      Dft<T, R0>::run(v);
    }
    __syncthreads();
    if (j < Q0) {
#pragma unroll
      for (int r = 0; r < R0; ++r) cur[(j * R0 + r) * TC + b] = v[r];
    }
    __syncthreads();
    if (j < Q1) {
#pragma unroll
      for (int r = 0; r < R1; ++r) v[r] = cur[(j + r * R0) * TC + b];
#pragma unroll
      for (int r = 1; r < R1; ++r) v[r] = cmul(v[r], __ldg(&tw[r * R0 + j]));
      Dft<T, R1>::run(v);
#pragma unroll
      for (int r = 0; r < R1; ++r) {
        T k = kmask_f<T, L>(jf + (T)(r * R0)) * sc;
        v[r] = mk<C>(-k * v[r].y, -k * v[r].x);
      }
      Dft<T, R1>::run(v);
    }
    __syncthreads();
    if (j < Q1) {
#pragma unroll
      for (int r = 0; r < R1; ++r) cur[(j * R1 + r) * TC + b] = v[r];
    }
    __syncthreads();
    if (j < Q0) {
#pragma unroll
      for (int r = 0; r < R0; ++r) v[r] = cur[(j + r * Q0) * TC + b];
#pragma unroll
      for (int r = 1; r < R0; ++r) v[r] = cmul(v[r], __ldg(&tw[j * R0 + r]));
      Dft<T, R0>::run(v);
#pragma unroll
      for (int r = 0; r < R0; ++r) {
        C z = cconj(v[r]);
        long o = off + (long)(j + r * Q0) * s + b;
        if (add) z = cadd(z, add[o]);
        out[o] = z;
      }
    }
    // the shared-memory writes above precede, in the async proxy, the tensor
    // copy that refills this buffer in the next iteration
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    __syncthreads();
    pending_other = false;
  }
  // after a timeout the copies issued for this and the next tile may still be
  // in flight: wait for them (bounded) before the block's shared memory is released
  if (t < ntiles) {
    (void)mbar_wait(&bar[it & 1], (it >> 1) & 1);
    if (pending_other) (void)mbar_wait(&bar[(it & 1) ^ 1], ((it + 1) >> 1) & 1);
  }
}


// ---------------------------------------------------------------------------
// Single-precision column passes of one stage in one persistent launch.
//
// Every thread transforms two neighbouring columns at once: a float2 holds
// the same quantity of both columns, and the butterflies run as paired
// single-precision instructions (add/fma/mul on float2, sm_100 and later),
// half the arithmetic instructions of one column per thread. Between the
// stages the tile lives in shared memory as two planes of column pairs
// (real parts, imaginary parts), so every exchange loads ready-made pairs.
//
// A launch covers up to four independent column passes (jobs) of the same
// axis length: each job has its own tensor map (input pencils), output,
// optional add, stride and tile count, and the blocks walk the
// concatenated tile list. One launch per stage replaces a launch per pass,
// so the ramp-up and the partial last wave of the persistent blocks are
// paid once per stage.
// ---------------------------------------------------------------------------
struct P2 {
  float2 re, im;
};
__device__ __forceinline__ P2 p2_add(P2 a, P2 b) { return {__fadd2_rn(a.re, b.re), __fadd2_rn(a.im, b.im)}; }
// a - b as a + (-1) b in one fused operation per half (exact: the product by -1 is not rounded)
__device__ __forceinline__ P2 p2_sub(P2 a, P2 b) {
  const float2 m1 = make_float2(-1.f, -1.f);
  return {__ffma2_rn(b.re, m1, a.re), __ffma2_rn(b.im, m1, a.im)};
}
// times the complex scalar (c, s), given as the duplicated pairs (c, c) and (s, s)
__device__ __forceinline__ P2 p2_mul(P2 a, float2 cc, float2 ss) {
  const float2 nss = __fmul2_rn(ss, make_float2(-1.f, -1.f));
  return {__ffma2_rn(a.re, cc, __fmul2_rn(a.im, nss)), __ffma2_rn(a.re, ss, __fmul2_rn(a.im, cc))};
}
template <int R, int k>
__device__ __forceinline__ P2 p2_twid(P2 o) {
  constexpr int q = (k * 16 / R) % 16;
  if constexpr (q == 0) return o;
  else if constexpr (q == 4) return {o.im, make_float2(-o.re.x, -o.re.y)};  // times -i
  else if constexpr (q == 8) return {make_float2(-o.re.x, -o.re.y), make_float2(-o.im.x, -o.im.y)};
  else if constexpr (q == 12) return {make_float2(-o.im.x, -o.im.y), o.re};  // times i
  else {
    const float2 w = root16<float, q>();
    return p2_mul(o, make_float2(w.x, w.x), make_float2(w.y, w.y));
  }
}
// forward DFT of size R on paired values (radix-2 decimation in time, as Dft)
template <int R>
struct P2Dft {
  template <int k>
  static __device__ __forceinline__ void comb(P2* v, const P2* e, const P2* o) {
    if constexpr (k < R / 2) {
      const P2 t = p2_twid<R, k>(o[k]);
      v[k] = p2_add(e[k], t);
      v[k + R / 2] = p2_sub(e[k], t);
      comb<k + 1>(v, e, o);
    }
  }
  static __device__ __forceinline__ void run(P2* v) {
    P2 e[R / 2], o[R / 2];
#pragma unroll
    for (int i = 0; i < R / 2; ++i) {
      e[i] = v[2 * i];
      o[i] = v[2 * i + 1];
    }
    P2Dft<R / 2>::run(e);
    P2Dft<R / 2>::run(o);
    comb<0>(v, e, o);
  }
};
template <>
struct P2Dft<1> {
  static __device__ __forceinline__ void run(P2*) {}
};

// float2 slot of (row, column pair cp) in one plane of 8 pairs per row; the
// rows of every odd 16-row group swap places pairwise, so the rows 16a + b
// that one store instruction touches fall on alternating halves of the banks
__device__ __forceinline__ int plane_slot(int row, int cp) { return ((row ^ ((row >> 4) & 1)) << 3) + cp; }

constexpr int kColJobs = 4;
struct ColJobs {
  float2* out[kColJobs];
  const float2* add[kColJobs];  // null: no add
  long s[kColJobs];             // stride between pencil elements (complex values)
  int ntx[kColJobs];            // tiles across the inner extent s / 16
  int start[kColJobs + 1];      // first global tile of each job; start[nj] = all tiles
  int rev[kColJobs];            // walk the job's tiles from the last one
  int nj;
};

// out = IFFT_a(i k~_a FFT_a(in)) (+ add) for the jobs' pencils of length
// L = R0 * R1, tiles of 16 columns, 8 column pairs x max(L/R0, R0) threads.
// Stages: A (radix R0) from the TMA tile, B (radix R1) with twiddles
// W_L^{r j}, the multiplier, the inverse first stage A' (radix R1) on the
// same registers, and B' (radix R0, twiddles read transposed) to global
// memory, as in k_cols_deriv2. tw2: the stage-1 twiddle block of length L
// with each entry (c, s) stored as (c, c, s, s).
template <int L, int R0, int R1>
__global__ void __launch_bounds__(8 * (L / R0 > R0 ? L / R0 : R0)) k_cols_pairs(
    const __grid_constant__ CUtensorMap m0, const __grid_constant__ CUtensorMap m1,
    const __grid_constant__ CUtensorMap m2, const __grid_constant__ CUtensorMap m3, ColJobs J,
    const float4* __restrict__ tw2) {
  constexpr int TC = 16;
  constexpr int Q0 = L / R0, Q1 = R0;
  constexpr unsigned TILE_BYTES = L * TC * sizeof(float2);
  constexpr int XW = TC * 2;  // box width in 4-byte elements
  constexpr int RMAX = R0 > R1 ? R0 : R1;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar[2];
  float2* bufs = reinterpret_cast<float2*>(smem_raw);  // two tiles of L x TC complex values
  const int cp = threadIdx.x & 7, j = threadIdx.x >> 3;
  const int ntiles = J.start[J.nj];
  auto job_of = [&](int tt) {
    int q = 0;
#pragma unroll
    for (int k = 1; k < kColJobs; ++k)
      if (k < J.nj && tt >= J.start[k]) q = k;
    return q;
  };
  auto local = [&](int tt, int q) {  // the job's own tile index of global tile tt
    const int lt = tt - J.start[q];
    return J.rev[q] ? J.start[q + 1] - J.start[q] - 1 - lt : lt;
  };
  auto issue = [&](int tt, int b) {  // one thread
    const int q = job_of(tt);
    const int lt = local(tt, q);
    const CUtensorMap* mp = q == 0 ? &m0 : (q == 1 ? &m1 : (q == 2 ? &m2 : &m3));
    mbar_expect_tx(&bar[b], TILE_BYTES);
    tma_load_2d(bufs + b * L * TC, mp, (lt % J.ntx[q]) * XW, (lt / J.ntx[q]) * L, &bar[b]);
  };
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  int t = blockIdx.x;
  if (threadIdx.x == 0 && t < ntiles) issue(t, 0);
  int it = 0;
  bool pending_other = false;  // a copy into the other buffer is in flight
  const float sc = 1.f / (float)L;
  P2 v[RMAX];
  for (; t < ntiles; t += gridDim.x, ++it) {
    const int cb = it & 1;
    float2* cur = bufs + cb * L * TC;
    float2* pre = cur;               // plane of real parts
    float2* pim = cur + L * TC / 2;  // plane of imaginary parts
    const int q = job_of(t);
    const int lt = local(t, q);
    const long s = J.s[q];
    const long off = (long)(lt / J.ntx[q]) * L * s + (long)(lt % J.ntx[q]) * TC;
    const int tn = t + gridDim.x;
    pending_other = tn < ntiles;
    if (threadIdx.x == 0 && pending_other) issue(tn, cb ^ 1);
    // all threads agree on the outcome, so a timeout ends the whole block together
    if (!__syncthreads_and(mbar_wait(&bar[cb], (it >> 1) & 1))) {
      if (threadIdx.x == 0) atomicAdd(&g_tma_timeouts, 1);
      break;
    }
    // forward stage A from the tile (complex values of columns 2cp, 2cp+1 are one float4)
    if (j < Q0) {
      const float4* c4 = reinterpret_cast<const float4*>(cur);
#pragma unroll
      for (int r = 0; r < R0; ++r) {
        const float4 x = c4[(j + r * Q0) * (TC / 2) + cp];
        v[r].re = make_float2(x.x, x.z);
        v[r].im = make_float2(x.y, x.w);
      }
      P2Dft<R0>::run(v);
    }
    __syncthreads();  // the tile has been read: its buffer now holds the planes
    if (j < Q0) {
#pragma unroll
      for (int r = 0; r < R0; ++r) {
        pre[plane_slot(j * R0 + r, cp)] = v[r].re;
        pim[plane_slot(j * R0 + r, cp)] = v[r].im;
      }
    }
    __syncthreads();
    if (j < Q1) {
#pragma unroll
      for (int r = 0; r < R1; ++r) {
        v[r].re = pre[plane_slot(j + r * R0, cp)];
        v[r].im = pim[plane_slot(j + r * R0, cp)];
      }
#pragma unroll
      for (int r = 1; r < R1; ++r) {
        const float4 w = __ldg(&tw2[r * R0 + j]);
        v[r] = p2_mul(v[r], make_float2(w.x, w.y), make_float2(w.z, w.w));
      }
      P2Dft<R1>::run(v);
      // v[r] is frequency j + r*R0: conj(i k~ z / L) = (-k z.im, -k z.re) with k = k~ / L
#pragma unroll
      for (int r = 0; r < R1; ++r) {
        const float k = kmask_f<float, L>((float)(j + r * R0)) * sc;
        const float2 nk = make_float2(-k, -k);
        const float2 re = __fmul2_rn(v[r].im, nk);
        v[r].im = __fmul2_rn(v[r].re, nk);
        v[r].re = re;
      }
      P2Dft<R1>::run(v);  // inverse stage A' on the same values
    }
    __syncthreads();  // every thread has read the planes of stage B
    if (j < Q1) {
#pragma unroll
      for (int r = 0; r < R1; ++r) {
        pre[plane_slot(j * R1 + r, cp)] = v[r].re;
        pim[plane_slot(j * R1 + r, cp)] = v[r].im;
      }
    }
    __syncthreads();
    if (j < Q0) {
#pragma unroll
      for (int r = 0; r < R0; ++r) {
        v[r].re = pre[plane_slot(j + r * Q0, cp)];
        v[r].im = pim[plane_slot(j + r * Q0, cp)];
      }
#pragma unroll
      for (int r = 1; r < R0; ++r) {
        const float4 w = __ldg(&tw2[j * R0 + r]);
        v[r] = p2_mul(v[r], make_float2(w.x, w.y), make_float2(w.z, w.w));
      }
      P2Dft<R0>::run(v);
      float2* out = J.out[q];
      const float2* add = J.add[q];
#pragma unroll
      for (int r = 0; r < R0; ++r) {
        float4 z = make_float4(v[r].re.x, -v[r].im.x, v[r].re.y, -v[r].im.y);  // conjugated back
        const long o = off + (long)(j + r * Q0) * s + 2 * cp;
        if (add) {
          const float4 a = *reinterpret_cast<const float4*>(add + o);
          z.x += a.x;
          z.y += a.y;
          z.z += a.z;
          z.w += a.w;
        }
        *reinterpret_cast<float4*>(out + o) = z;
      }
    }
    // the shared-memory writes above precede, in the async proxy, the tensor
    // copy that refills this buffer in the next iteration
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    __syncthreads();
    pending_other = false;
  }
  // after a timeout the copies issued for this and the next tile may still be
  // in flight: wait for them (bounded) before the block's shared memory is released
  if (t < ntiles) {
    (void)mbar_wait(&bar[it & 1], (it >> 1) & 1);
    if (pending_other) (void)mbar_wait(&bar[(it & 1) ^ 1], ((it + 1) >> 1) & 1);
  }
}

}  // namespace fused
}  // namespace reg
