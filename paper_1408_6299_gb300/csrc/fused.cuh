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
#include "internal.h"

namespace reg {
namespace fused {

constexpr int kThreads = 256;

__host__ __device__ inline long kmask_l(long j, long n) { return j == n / 2 ? 0 : (j < n / 2 ? j : j - n); }

template <typename T, int NF>
struct RowsIn {
  const T* p[NF];
};
template <typename T, int NF>
struct RowsOut {
  cx<T>* p[NF];
};

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
  for (int e = threadIdx.x; e < NF * RB * M; e += kThreads) {
    int f = e / (RB * M), rem = e % (RB * M);
    int r = rem / M, j = rem % M;
    long row = row0 + r;
    C z = mk<C>(0, 0);
    if (row < nrows) {
      z = reinterpret_cast<const C*>(in.p[f])[row * M + j];
      if (PROD) {
        C l = reinterpret_cast<const C*>(lam)[row * M + j];
        z = mk<C>(z.x * l.x, z.y * l.y);
      }
    }
    buf[(f * RB + r) * RS + pad16(j)] = z;
  }
  __syncthreads();
  smem_fft<T, M, false, kThreads, NF * RB>(buf, RS, tw);
  constexpr int H = M / 2 + 1;
  for (int e = threadIdx.x; e < NF * RB * H; e += kThreads) {
    int seq = e / H, k = e % H;
    int f = seq / RB, r = seq % RB;
    long row = row0 + r;
    if (row >= nrows) continue;
    C* o = out.p[f] + row * M;
    const C* b = buf + seq * RS;
    bool dz = (zmask >> f) & 1;
    if (k == 0) {
      C z0 = b[0];
      o[0] = dz ? mk<C>(0, 0) : mk<C>(z0.x + z0.y, z0.x - z0.y);
    } else {
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
    }
  }
}

// Epilogue parameters of the advection stage (state / incremental state).
template <typename T>
struct AdvEpi {
  const T* a[3];   // velocity components at the stage time
  const T* gm[3];  // source: grad m at the stage time (null: no source)
  const T* w[3];   // source: incremental velocity at the stage time
  const T* y;      // stage 1: y_j (null = 0); stage 2: acc
  T* out1;         // stage 1: y_j + h k; stage 2: acc + h/2 k
  T* out2;         // stage 1: y_j + h/2 k
  T* G[3];         // optional: keep grad u (null: not stored)
  T h;
  int stage;
};

// Epilogue parameters of the divergence stage (adjoint / incremental adjoint).
template <typename T>
struct DivEpi {
  const T* y;  // stage 1: lam_{j+1}; stage 2: acc
  T* out1;
  T* out2;
  T h;
  int stage;
};

template <typename T, int NF>
struct RowsSpec {
  const cx<T>* p[NF];
};

enum { EPI_ADV = 1, EPI_DIV = 2 };

// Complex-to-real rows of NF fields, then the stage epilogue on the real
// values (each thread handles a pair of neighbouring points). Fields whose
// bit is set in zmask are multiplied by i k_last on load.
template <typename T, int L, int RB, int NF, int EPI>
__global__ void __launch_bounds__(kThreads) k_rows_c2r_n(RowsSpec<T, NF> in, int zmask, AdvEpi<T> adv,
                                                          DivEpi<T> dv, long nrows, const cx<T>* __restrict__ tw,
                                                          const cx<T>* __restrict__ twrc) {
  using C = cx<T>;
  constexpr int M = L / 2;
  constexpr int RS = padded_len(M);
  __shared__ C buf[NF * RB * RS];
  const long row0 = (long)blockIdx.x * RB;
  for (int e = threadIdx.x; e < NF * RB * M; e += kThreads) {
    int f = e / (RB * M), rem = e % (RB * M);
    int r = rem / M, j = rem % M;
    long row = row0 + r;
    C z = mk<C>(0, 0);
    if (row < nrows) {
      z = in.p[f][row * M + j];
      if ((zmask >> f) & 1) z = mk<C>(-(T)j * z.y, (T)j * z.x);
    }
    buf[(f * RB + r) * RS + pad16(j)] = z;
  }
  __syncthreads();
  constexpr int H = M / 2 + 1;
  for (int e = threadIdx.x; e < NF * RB * H; e += kThreads) {
    int seq = e / H, k = e % H;
    C* b = buf + seq * RS;
    if (k == 0) {
      C p = b[0];
      b[0] = cconj(mk<C>((p.x + p.y) * (T)0.5, (p.x - p.y) * (T)0.5));
    } else {
      C xk = b[pad16(k)], xm = b[pad16(M - k)];
      C E = cscale(cadd(xk, cconj(xm)), (T)0.5);
      C Od = cscale(cmul(csub(xk, cconj(xm)), cconj(__ldg(&twrc[k]))), (T)0.5);
      C zk = mk<C>(E.x - Od.y, E.y + Od.x);
      C zm = mk<C>(E.x + Od.y, -E.y + Od.x);
      b[pad16(k)] = cconj(zk);
      if (k != M - k) b[pad16(M - k)] = cconj(zm);
    }
  }
  __syncthreads();
  smem_fft<T, M, false, kThreads, NF * RB>(buf, RS, tw);
  const T s = (T)1 / (T)M;
  for (int e = threadIdx.x; e < RB * M; e += kThreads) {
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
      if (adv.G[0]) {
#pragma unroll
        for (int f = 0; f < NF; ++f) reinterpret_cast<C*>(adv.G[f])[q] = g[f];
      }
      T k0 = 0, k1 = 0;
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        C a = reinterpret_cast<const C*>(adv.a[f])[q];
        k0 -= a.x * g[f].x;
        k1 -= a.y * g[f].y;
      }
      if (adv.gm[0]) {
#pragma unroll
        for (int f = 0; f < NF; ++f) {
          C gm = reinterpret_cast<const C*>(adv.gm[f])[q];
          C w = reinterpret_cast<const C*>(adv.w[f])[q];
          k0 -= gm.x * w.x;
          k1 -= gm.y * w.y;
        }
      }
      if (adv.stage == 1) {
        C yv = adv.y ? reinterpret_cast<const C*>(adv.y)[q] : mk<C>(0, 0);
        reinterpret_cast<C*>(adv.out1)[q] = mk<C>(yv.x + adv.h * k0, yv.y + adv.h * k1);
        reinterpret_cast<C*>(adv.out2)[q] = mk<C>(yv.x + (T)0.5 * adv.h * k0, yv.y + (T)0.5 * adv.h * k1);
      } else {
        C yv = reinterpret_cast<const C*>(adv.y)[q];
        reinterpret_cast<C*>(adv.out1)[q] = mk<C>(yv.x + (T)0.5 * adv.h * k0, yv.y + (T)0.5 * adv.h * k1);
      }
    } else {
      C k = g[0];
      C yv = reinterpret_cast<const C*>(dv.y)[q];
      if (dv.stage == 1) {
        reinterpret_cast<C*>(dv.out1)[q] = mk<C>(yv.x + dv.h * k.x, yv.y + dv.h * k.y);
        reinterpret_cast<C*>(dv.out2)[q] = mk<C>(yv.x + (T)0.5 * dv.h * k.x, yv.y + (T)0.5 * dv.h * k.y);
      } else {
        reinterpret_cast<C*>(dv.out1)[q] = mk<C>(yv.x + (T)0.5 * dv.h * k.x, yv.y + (T)0.5 * dv.h * k.y);
      }
    }
  }
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
  for (int e = threadIdx.x; e < L * TC; e += kThreads) {
    int j = e / TC, c = e % TC;
    buf[j * TC + c] = in[off + (long)j * s + c];
  }
  __syncthreads();
  smem_fft<T, L, true, kThreads, TC>(buf, TC, tw);
  const T sc = (T)1 / (T)L;
  for (int e = threadIdx.x; e < L * TC; e += kThreads) {
    int j = e / TC;
    T k = (T)kmask_l(j, L) * sc;
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

}  // namespace fused
}  // namespace reg
