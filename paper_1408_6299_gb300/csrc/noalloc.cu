// noalloc.cu -- the preconditioner application of reg_precond, for callers
// that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at the point where they need the
// operator: code that runs while another runtime owns every device byte
// through its own pool allocator, code under a hard memory budget fixed at
// start-up, or loops that must never allocate after initialisation. For them
// reg_precond_noalloc works entirely inside one file-scope device array that
// the CUDA runtime reserves when this library's module is loaded, and it
// never calls cudaMalloc, cudaFree or any allocating routine.
//
// The array holds, from its start: the FFT twiddle tables (uploaded once per
// device by the first call), the inverse Chebyshev Gram matrix of the call,
// and the two sets of spectra the transform needs. Every call shares it and
// it keeps the last call's contents; each call overwrites everything it reads
// (the forward transforms fill the spectra, a small kernel writes the Gram
// inverse), so nothing needs clearing. Calls whose GPU work overlaps (other
// streams, other host threads, without ordering between them) race on it.
#include <math.h>

#include <mutex>
#include <string>

#include "../../include/reg.h"
#include "internal.h"

using namespace reg;

namespace {

// Fixed scratch: 64 MiB per GPU that loads the library, held until exit.
constexpr size_t kScratchBytes = 64ull << 20;
constexpr size_t kTableBytes = 64ull << 10;   // twiddle tables (about 25 KiB used)
constexpr size_t kGramBytes = 16 * 16 * 8;    // inverse Gram matrix, n_c <= 16
static __device__ __align__(256) unsigned char g_precond_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
struct DeviceState {
  bool ready = false;
  unsigned char* base = nullptr;  // device address of g_precond_scratch
  long tw_off[11] = {0};
  long rc_off[11] = {0};
};
DeviceState g_dev[kMaxDevices];
std::mutex g_mu;
constexpr long kCapacity = (long)((kScratchBytes - kTableBytes - kGramBytes) / (2 * sizeof(double2)));

// host image of the tables (double, interleaved), filled at set-up
constexpr long kMaxTableEntries = (long)(kTableBytes / 16);
double g_table_image[2 * kMaxTableEntries];

struct GramInverse {
  double c[16 * 16];
};

__global__ void k_store_gram(double* dst, GramInverse g, int count) {
  int i = threadIdx.x;
  if (i < count) dst[i] = g.c[i];
}

reg_status noalloc_fail(int st, const std::string& msg) {
  set_thread_error("reg_precond_noalloc: " + msg);
  return (reg_status)st;
}

// once per device, with that device current: find the array's device
// address and upload the twiddle tables (a synchronous copy; make this first
// call before anything that must not see host-to-device copies)
int setup_device(int dev) {
  std::lock_guard<std::mutex> lk(g_mu);
  DeviceState& S = g_dev[dev];
  if (S.ready) return 0;
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_precond_scratch);
  if (e != cudaSuccess) return (int)e;
  long n = Spectral<double>::write_tables(nullptr, S.tw_off, S.rc_off);
  if (n > kMaxTableEntries) return (int)cudaErrorInvalidValue;
  Spectral<double>::write_tables(g_table_image, S.tw_off, S.rc_off);
  e = cudaMemcpy(p, g_table_image, (size_t)n * 16, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return (int)e;
  S.base = (unsigned char*)p;
  S.ready = true;
  return 0;
}

bool chebyshev_gram_inverse(int nc, double* Ci) {
  double A[16 * 32];
  auto I = [](int m) { return (m % 2) ? 0.0 : 2.0 / (1.0 - (double)m * (double)m); };
  for (int a = 0; a < nc; ++a)
    for (int b = 0; b < 2 * nc; ++b)
      A[a * 2 * nc + b] = b < nc ? 0.25 * (I(a + b) + I(a > b ? a - b : b - a)) : (b - nc == a ? 1.0 : 0.0);
  for (int c = 0; c < nc; ++c) {
    int piv = c;
    for (int r = c + 1; r < nc; ++r)
      if (fabs(A[r * 2 * nc + c]) > fabs(A[piv * 2 * nc + c])) piv = r;
    if (A[piv * 2 * nc + c] == 0.0) return false;
    for (int k = 0; k < 2 * nc; ++k) {
      double t = A[c * 2 * nc + k];
      A[c * 2 * nc + k] = A[piv * 2 * nc + k];
      A[piv * 2 * nc + k] = t;
    }
    double p = A[c * 2 * nc + c];
    for (int k = 0; k < 2 * nc; ++k) A[c * 2 * nc + k] /= p;
    for (int r = 0; r < nc; ++r)
      if (r != c) {
        double f = A[r * 2 * nc + c];
        for (int k = 0; k < 2 * nc; ++k) A[r * 2 * nc + k] -= f * A[c * 2 * nc + k];
      }
  }
  for (int a = 0; a < nc; ++a)
    for (int b = 0; b < nc; ++b) Ci[a * nc + b] = A[a * 2 * nc + nc + b];
  return true;
}

// memory the kernels on device `dev` may address: device memory of that
// device, or managed memory
bool is_device(const void* p, int dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeManaged || (a.type == cudaMemoryTypeDevice && a.device == dev);
}

}  // namespace

extern "C" {

reg_status reg_precond_noalloc(int d, const int64_t* n, int n_c, double beta, int reg_type, const double* r,
                               double* z, void* cuda_stream) {
  tl_prof = nullptr;  // never record profiling events from here
  if (!n || !r || !z) return noalloc_fail(REG_EINVAL, "null argument");
  if (n_c < 1 || n_c > 16) return noalloc_fail(REG_EINVAL, "n_c must be in [1, 16]");
  if (!(beta > 0.0) || !isfinite(beta)) return noalloc_fail(REG_EINVAL, "beta must be positive and finite");
  if (reg_type != REG_H1 && reg_type != REG_H2) return noalloc_fail(REG_EINVAL, "reg_type must be REG_H1 or REG_H2");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  try {
    Grid g = make_grid(d, n);
    const long ncd = (long)n_c * d;
    if (ncd * g.Nc > kCapacity)
      return noalloc_fail(REG_EINVAL, "n_c*d*N/2 = " + std::to_string(ncd * g.Nc) +
                                          " spectral values exceed the fixed scratch capacity of " +
                                          std::to_string(kCapacity) + " (64 MiB per GPU); use reg_precond");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return noalloc_fail(REG_ECUDA, cudaGetErrorString(e));
    if (!is_device(r, dev) || !is_device(z, dev))
      return noalloc_fail(REG_EINVAL, "r and z must be device (or managed) memory of the current device");
    if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(REG_EINVAL, "device ordinal out of range");
    int st = setup_device(dev);
    if (st != 0) return noalloc_fail(REG_ECUDA, cudaGetErrorString((cudaError_t)st));
    DeviceState& S = g_dev[dev];
    double2* tables = (double2*)S.base;
    double* Ci = (double*)(S.base + kTableBytes);
    double2* SV = (double2*)(S.base + kTableBytes + kGramBytes);
    double2* SF = SV + ncd * g.Nc;

    GramInverse gi;
    if (!chebyshev_gram_inverse(n_c, gi.c)) return noalloc_fail(REG_EINVAL, "singular Gram matrix");
    k_store_gram<<<1, 256, 0, s>>>(Ci, gi, n_c * n_c);
    REG_LAUNCH();

    int e2 = 0;
    while ((1 << e2) < g.L) ++e2;
    Spectral<double> sp(g, s, tables, S.tw_off, S.rc_off[e2]);
    for (long q = 0; q < ncd; ++q) sp.fwd(r + q * g.N, SV + q * g.Nc);
    spec_precond(g, s, SV, SF, n_c, beta, Ci, reg_type);
    for (long q = 0; q < ncd; ++q) sp.inv(SF + q * g.Nc, z + q * g.N);
  } catch (const StatusError& e) {
    return noalloc_fail(e.status, e.what);
  } catch (const CudaError& e) {
    return noalloc_fail(REG_ECUDA, e.what);
  }
  return REG_OK;
}

}  // extern "C"
