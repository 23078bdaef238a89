// fft.cuh -- device building blocks of the power-of-two FFTs behind the Fourier
// pseudospectral operators (Mang & Biros, Sec. 3.3.1: derivatives by Fourier
// spectral methods on a periodic nodal grid).
//
// Conventions: forward transform X[k] = sum_j x[j] exp(-2 pi i jk/L), inverse
// with exp(+2 pi i jk/L) and 1/L. Inverse transforms are formed as
// conj(FFT(conj(x))), so only forward butterflies exist. Twiddles come from
// tables computed on the host in double precision and rounded once.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace reg {

template <typename T> struct Cx;
template <> struct Cx<float> { using type = float2; };
template <> struct Cx<double> { using type = double2; };
template <typename T> using cx = typename Cx<T>::type;

template <typename C> __device__ __forceinline__ C mk(decltype(C::x) a, decltype(C::x) b) {
  C c;
  c.x = a;
  c.y = b;
  return c;
}
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return mk<C>(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return mk<C>(a.x - b.x, a.y - b.y); }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  return mk<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename C> __device__ __forceinline__ C cconj(C a) { return mk<C>(a.x, -a.y); }
// multiply by -i
template <typename C> __device__ __forceinline__ C cmul_mi(C a) { return mk<C>(a.y, -a.x); }
template <typename C> __device__ __forceinline__ C cscale(C a, decltype(C::x) s) { return mk<C>(a.x * s, a.y * s); }

// exp(-2 pi i q/16) for compile-time q in [0,16): the 16th roots of unity.
// cos(pi/8) and sin(pi/8) written out; sqrt(1/2) likewise.
// The constants are rounded to T at compile time, so a single-precision
// butterfly issues no double-precision conversion.
template <typename T, int q> __device__ __forceinline__ cx<T> root16() {
  constexpr T c1 = (T)0.92387953251128675613;  // cos(pi/8)
  constexpr T s1 = (T)0.38268343236508977173;  // sin(pi/8)
  constexpr T h = (T)0.70710678118654752440;   // sqrt(1/2)
  constexpr T o = (T)1, z = (T)0;
  constexpr T re[16] = {o, c1, h, s1, z, -s1, -h, -c1, -o, -c1, -h, -s1, z, s1, h, c1};
  constexpr T im[16] = {z, -s1, -h, -c1, -o, -c1, -h, -s1, z, s1, h, c1, o, c1, h, s1};
  constexpr T a = re[q], b = im[q];
  return mk<cx<T>>(a, b);
}

// o * exp(-2 pi i k / R) with compile-time k, R <= 16; trivial roots skip the multiply.
template <typename T, int R, int k> __device__ __forceinline__ cx<T> twid_const(cx<T> o) {
  constexpr int q = (k * 16 / R) % 16;
  if constexpr (q == 0) return o;
  else if constexpr (q == 4) return cmul_mi(o);
  else if constexpr (q == 8) return mk<cx<T>>(-o.x, -o.y);
  else if constexpr (q == 12) return mk<cx<T>>(-o.y, o.x);
  else return cmul(o, root16<T, q>());
}

// e + t and e - t of one radix-2 butterfly. Single precision issues each as
// one paired instruction (sm_100 and later; e - t as e + (-1) t, exact),
// the same roundings as the componentwise form. Twiddles that are multiples
// of -i (a swap and a sign) keep the componentwise form, where the sign
// folds into the addition.
template <typename T, int q>
__device__ __forceinline__ void bfly(cx<T> e, cx<T> t, cx<T>& a, cx<T>& b) {
  if constexpr (sizeof(T) == 4 && (q == 0 || q % 4 != 0)) {
    a = __fadd2_rn(e, t);
    b = __ffma2_rn(t, make_float2(-1.f, -1.f), e);
  } else {
    a = cadd(e, t);
    b = csub(e, t);
  }
}

// In-register forward DFT of size R (power of two, R <= 16): radix-2
// decimation in time, recursively.
template <typename T, int R> struct Dft {
  template <int k> static __device__ __forceinline__ void comb(cx<T>* v, const cx<T>* e, const cx<T>* o) {
    if constexpr (k < R / 2) {
      cx<T> t = twid_const<T, R, k>(o[k]);
      bfly<T, (k * 16 / R) % 16>(e[k], t, v[k], v[k + R / 2]);
      comb<k + 1>(v, e, o);
    }
  }
  static __device__ __forceinline__ void run(cx<T>* v) {
    cx<T> e[R / 2], o[R / 2];
#pragma unroll
    for (int i = 0; i < R / 2; ++i) {
      e[i] = v[2 * i];
      o[i] = v[2 * i + 1];
    }
    Dft<T, R / 2>::run(e);
    Dft<T, R / 2>::run(o);
    comb<0>(v, e, o);
  }
};
template <typename T> struct Dft<T, 1> {
  static __device__ __forceinline__ void run(cx<T>*) {}
};

// ---------------------------------------------------------------------------
// Radix plans: L = R0 * R1 * ...; stage s has Ns = R0*...*R_{s-1}.
// ---------------------------------------------------------------------------
template <int L> struct Plan;
template <> struct Plan<2> { static constexpr int S = 1; static constexpr int R[3] = {2, 1, 1}; };
template <> struct Plan<4> { static constexpr int S = 1; static constexpr int R[3] = {4, 1, 1}; };
template <> struct Plan<8> { static constexpr int S = 1; static constexpr int R[3] = {8, 1, 1}; };
template <> struct Plan<16> { static constexpr int S = 1; static constexpr int R[3] = {16, 1, 1}; };
template <> struct Plan<32> { static constexpr int S = 2; static constexpr int R[3] = {8, 4, 1}; };
template <> struct Plan<64> { static constexpr int S = 2; static constexpr int R[3] = {8, 8, 1}; };
template <> struct Plan<128> { static constexpr int S = 2; static constexpr int R[3] = {16, 8, 1}; };
template <> struct Plan<256> { static constexpr int S = 2; static constexpr int R[3] = {16, 16, 1}; };
template <> struct Plan<512> { static constexpr int S = 3; static constexpr int R[3] = {8, 8, 8}; };

// Real floating-point operations of Dft<T,R>::run: two half-size DFTs, R
// complex additions and one complex multiplication (6 operations) per
// constant twiddle that is not a multiple of -i.
__host__ __device__ constexpr double dft_flops(int R) {
  if (R <= 1) return 0.0;
  int general = 0;
  for (int k = 0; k < R / 2; ++k)
    if (((k * 16 / R) % 16) % 4 != 0) ++general;
  return 2.0 * dft_flops(R / 2) + 2.0 * R + 6.0 * general;
}

// Real floating-point operations of one forward transform of length L along
// the radix plan: the butterflies of every stage and the complex twiddle
// multiplications between stages (counted for every stage after the first,
// trivial table entries included, as the kernels execute them).
template <int L>
constexpr double fft_flops() {
  using P = Plan<L>;
  double f = 0.0;
  for (int s = 0; s < P::S; ++s) {
    f += (double)(L / P::R[s]) * dft_flops(P::R[s]);
    if (s > 0) f += (double)(L / P::R[s]) * (P::R[s] - 1) * 6.0;
  }
  return f;
}

// Offset of stage s's twiddle block inside the table of length L. Stage s
// (radix R, Ns previous) stores W_{Ns R}^{r k} at [r*Ns + k], r < R, k < Ns.
// Stage 0 needs none.
__host__ __device__ constexpr int stage_tw_offset(int L, int s) {
  // blocks of stages 1..s-1 come first; each block of stage t has R_t*Ns_t = Ns_{t+1} entries
  int off = 0, ns = 1;
  int r[3] = {0, 0, 0};
  if (L == 2) { r[0] = 2; }
  else if (L == 4) { r[0] = 4; }
  else if (L == 8) { r[0] = 8; }
  else if (L == 16) { r[0] = 16; }
  else if (L == 32) { r[0] = 8; r[1] = 4; }
  else if (L == 64) { r[0] = 8; r[1] = 8; }
  else if (L == 128) { r[0] = 16; r[1] = 8; }
  else if (L == 256) { r[0] = 16; r[1] = 16; }
  else if (L == 512) { r[0] = 8; r[1] = 8; r[2] = 8; }
  for (int t = 0; t < s; ++t) {
    if (t > 0) off += ns * r[t];
    ns *= r[t];
  }
  return off;
}

// Padded shared-memory index: one spare slot after every 16 elements keeps
// strided stage stores free of bank conflicts for 8- and 16-byte elements.
__device__ __forceinline__ int pad16(int i) { return i + (i >> 4); }
__host__ __device__ constexpr int padded_len(int n) { return n + n / 16; }

// One forward radix-R Stockham stage (natural order in, natural order out),
// in place in shared memory, on B sequences of length L.
//   element j of sequence b lives at buf[b*bs + pad16(j)] (ROWS layout) or at
//   buf[j*bs + b] (COLS layout, bs = number of columns; neighbouring threads
//   take neighbouring columns, so no padding is needed there).
// Every thread loads all its butterflies into registers, the block
// synchronises, then the results are stored; a second barrier follows.
template <typename T, int L, int R, int NS, bool COLS, int NT, int B>
__device__ __forceinline__ void stockham_stage(cx<T>* buf, int bs, const cx<T>* __restrict__ tw) {
  constexpr int Q = L / R;  // butterflies per sequence
  constexpr int tasks = B * Q;
  constexpr int MAXT = (tasks + NT - 1) / NT;  // butterflies held per thread
  cx<T> v[MAXT][R];
  int nmine = 0;
#pragma unroll
  for (int it = 0; it < MAXT; ++it) {
    int t = threadIdx.x + it * NT;
    if (t < tasks) {
      int b = COLS ? (t % B) : (t / Q);
      int j = COLS ? (t / B) : (t % Q);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        int e = j + r * Q;
        v[it][r] = COLS ? buf[e * bs + b] : buf[b * bs + pad16(e)];
      }
      if constexpr (NS > 1) {
        int k = j % NS;
#pragma unroll
        for (int r = 1; r < R; ++r) v[it][r] = cmul(v[it][r], __ldg(&tw[r * NS + k]));
      }
      Dft<T, R>::run(v[it]);
      nmine = it + 1;
    }
  }
  __syncthreads();
#pragma unroll
  for (int it = 0; it < MAXT; ++it) {
    if (it < nmine) {
      int t = threadIdx.x + it * NT;
      int b = COLS ? (t % B) : (t / Q);
      int j = COLS ? (t / B) : (t % Q);
      int base = (j / NS) * NS * R + (j % NS);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        int e = base + r * NS;
        if (COLS) buf[e * bs + b] = v[it][r];
        else buf[b * bs + pad16(e)] = v[it][r];
      }
    }
  }
  __syncthreads();
}

// Full forward FFT of length L on B (compile-time) sequences held in shared memory.
// tw: device table for length L (stage blocks, see stage_tw_offset).
template <typename T, int L, bool COLS, int NT, int B>
__device__ __forceinline__ void smem_fft(cx<T>* buf, int bs, const cx<T>* __restrict__ tw) {
  using P = Plan<L>;
  constexpr int R0 = P::R[0], R1 = P::R[1], R2 = P::R[2];
  stockham_stage<T, L, R0, 1, COLS, NT, B>(buf, bs, tw);
  if constexpr (P::S > 1) stockham_stage<T, L, R1, R0, COLS, NT, B>(buf, bs, tw + stage_tw_offset(L, 1));
  if constexpr (P::S > 2) stockham_stage<T, L, R2, R0 * R1, COLS, NT, B>(buf, bs, tw + stage_tw_offset(L, 2));
}

}  // namespace reg
