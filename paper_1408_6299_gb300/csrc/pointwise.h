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

}  // namespace reg
