// fused_launch.cuh -- host launchers of the fused transport stages
// (fused.cuh), instantiated once per precision by fused_f32.cu / fused_f64.cu.
#pragma once
#include <stdlib.h>

#include <map>
#include <mutex>
#include <string>
#include <tuple>

#include "fused.cuh"

namespace reg {
namespace fused {

constexpr int pow2_ceil(int n) { return n <= 1 ? 1 : (n <= 2 ? 2 : 4); }

// complex values per block of the row passes
template <typename T>
constexpr int row_elems() {
  return sizeof(T) == 4 ? 4096 : 2048;
}

// Single-precision real-to-complex row passes on the edge-stage transforms
// (two-stage plans, last axis 64, 128 or 256) unless REG_EDGE_ROWS=0.
inline bool edge_rows_enabled() {
  static const bool on = [] {
    const char* env = getenv("REG_EDGE_ROWS");
    return !(env && env[0] == '0');
  }();
  return on;
}
// blocks of kernel `kern` (nt threads, smem dynamic bytes) resident on the
// whole current device at once
template <typename K>
int persistent_wave(K kern, int nt, size_t smem) {
  REG_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0, dev = 0, sms = 0;
  REG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, nt, smem));
  REG_CUDA(cudaGetDevice(&dev));
  REG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  return (per_sm < 1 ? 1 : per_sm) * sms;
}

// threads of an edge real-to-complex block: one first-stage butterfly each
template <int M, int NF, int RB>
constexpr int edge_r2c_threads() {
  return (NF * RB * Edge<M>::R1 + 31) / 32 * 32;
}
template <typename T, int L, int NF, bool PROD, int RB>
void r2c_launch(const Grid& g, cudaStream_t s, const RowsIn<T, NF>& in, const T* lam, const RowsOut<T, NF>& out,
                int zmask, const cx<T>* tw, const cx<T>* twrc) {
  dim3 grid((unsigned)((g.rows + RB - 1) / RB));
  if constexpr (sizeof(T) == 4 && Edge<L / 2>::ok) {  // double precision: FP64-pipe-bound, staged kernel
    if (edge_rows_enabled()) {
      constexpr int NT = edge_r2c_threads<L / 2, NF, RB>();
      k_rows_r2c_e<T, L, RB, NF, PROD, NT><<<grid, NT, 0, s>>>(in, lam, out, zmask, g.rows, tw, twrc);
      REG_LAUNCH();
      return;
    }
  }
  k_rows_r2c_n<T, L, RB, NF, PROD><<<grid, kThreads, 0, s>>>(in, lam, out, zmask, g.rows, tw, twrc);
  REG_LAUNCH();
}

// Choice of the autotuner among variants 0..nv-1 of a pure pass (one that
// writes only what it does not read, so running it again gives the same
// result): the persistent or per-process choice for `key`, else, outside a
// stream capture, each variant runs three times on the call's own buffers,
// timed with CUDA events on the stream, after one untimed run of each; the
// fastest is recorded. During a capture the first variant is used untuned.
template <typename Run>
int tuned_choice(const std::string& key, int nv, cudaStream_t st, Run run) {
  static std::mutex mu;
  static std::map<std::string, int> mem;
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = mem.find(key);
    if (it != mem.end()) return it->second;
  }
  int pick = tune_lookup(key);
  if (pick < 0 || pick >= nv) {
    const char* env = getenv("REG_AUTOTUNE");
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    REG_CUDA(cudaStreamIsCapturing(st, &cs));
    if ((env && env[0] == '0') || cs != cudaStreamCaptureStatusNone) return 0;
    cudaEvent_t e0, e1;
    REG_CUDA(cudaEventCreate(&e0));
    REG_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    pick = 0;
    for (int v = 0; v < nv; ++v) run(v);
    for (int v = 0; v < nv; ++v) {
      float total = 0;
      for (int r = 0; r < 3; ++r) {
        REG_CUDA(cudaEventRecord(e0, st));
        run(v);
        REG_CUDA(cudaEventRecord(e1, st));
        REG_CUDA(cudaEventSynchronize(e1));
        float ms = 0;
        REG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        total += ms;
      }
      if (total < best) {
        best = total;
        pick = v;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    tune_store(key, pick);
  }
  std::lock_guard<std::mutex> lk(mu);
  mem[key] = pick;
  return pick;
}

template <typename T, int L, int NF, bool PROD>
void r2c_L(const Grid& g, cudaStream_t s, const RowsIn<T, NF>& in, const T* lam, const RowsOut<T, NF>& out, int zmask,
           const cx<T>* tw, const cx<T>* twrc) {
  constexpr int M = L / 2;
  // single precision, one field: 2048 complex values per block (16 rows at L = 256) measured best
  // against 1024 and 8192 on the 256^3 matvec; the autotuner also tries half as many rows per block
  constexpr int RB0 = row_elems<T>() / (pow2_ceil(NF) * M * (sizeof(T) == 4 && NF == 1 ? 2 : 1));
  constexpr int RB = RB0 < 1 ? 1 : RB0;
  constexpr int RBh = RB > 1 ? RB / 2 : 1;
  ProfScope ps(KK_ROWS_R2C, s, (double)g.N * sizeof(T) * (2 * NF + (PROD ? 1 : 0)),
               (double)g.rows * NF * (fft_flops<M>() + 8.0 * M));
  auto run = [&](int v) {
    if (v == 0) r2c_launch<T, L, NF, PROD, RB>(g, s, in, lam, out, zmask, tw, twrc);
    else r2c_launch<T, L, NF, PROD, RBh>(g, s, in, lam, out, zmask, tw, twrc);
  };
  int v = 0;
  if (RBh != RB) {
    long rb = 1;  // row count rounded up to a power of two: stacks of similar size share a choice
    while (rb < g.rows) rb *= 2;
    const std::string key = tune_device_tag() + "|rows_r2c|" + (sizeof(T) == 4 ? "f32" : "f64") + "|L" +
                            std::to_string(L) + "|nf" + std::to_string(NF) + (PROD ? "p" : "") + "|rows" +
                            std::to_string(rb);
    v = tuned_choice(key, 2, s, run);
  }
  run(v);
}

template <typename T, int NF, bool PROD>
void r2c(const Grid& g, cudaStream_t s, const RowsIn<T, NF>& in, const T* lam, const RowsOut<T, NF>& out, int zmask,
         const cx<T>* tw, const cx<T>* twrc) {
  switch (g.L) {
    case 8: return r2c_L<T, 8, NF, PROD>(g, s, in, lam, out, zmask, tw, twrc);
    case 16: return r2c_L<T, 16, NF, PROD>(g, s, in, lam, out, zmask, tw, twrc);
    case 32: return r2c_L<T, 32, NF, PROD>(g, s, in, lam, out, zmask, tw, twrc);
    case 64: return r2c_L<T, 64, NF, PROD>(g, s, in, lam, out, zmask, tw, twrc);
    case 128: return r2c_L<T, 128, NF, PROD>(g, s, in, lam, out, zmask, tw, twrc);
    case 256: return r2c_L<T, 256, NF, PROD>(g, s, in, lam, out, zmask, tw, twrc);
    case 512: return r2c_L<T, 512, NF, PROD>(g, s, in, lam, out, zmask, tw, twrc);
  }
  throw StatusError{1, "unsupported last-axis length"};
}

template <typename T, int L, int NF, int EPI, int NE>
void c2r_L(const Grid& g, cudaStream_t s, const RowsSpec<T, NF>& in, int zmask, const AdvEpi<T>& adv,
           const DivEpi<T>& dv, double bytes, const cx<T>* tw, const cx<T>* twrc, const AdvEpi<T>& advB,
           const Emit<T>& em) {
  constexpr int M = L / 2;
  // single precision: 512 complex values per field and block for one field,
  // 1024 for more (4 and 8 rows at L = 256), so that the epilogue operand
  // slices stay within the prefetch limit (measured on the 256^3 matvec:
  // 298 -> 290 ms against the element-count rule of the other passes); the
  // emitting pass (NE = 1) takes 4 rows at L = 256 (222.5 -> 220.4 ms against 8)
  constexpr int NX = EPI == EPI_DIVS ? 1 : NF;  // sequences transformed per row
  constexpr int RB0 = sizeof(T) == 4 ? row_elems<T>() / ((NX == 1 || NX > 4 || NE > 0 ? 8 : 4) * M)
                                     : row_elems<T>() / ((NX > 4 ? 8 : pow2_ceil(NX)) * M);
  constexpr int RB = RB0 < 1 ? 1 : RB0;
  ProfScope ps(KK_ROWS_C2R, s, bytes, (double)g.rows * (NX + NE) * (fft_flops<M>() + 8.0 * M));
  dim3 grid((unsigned)((g.rows + RB - 1) / RB));
  k_rows_c2r_n<T, L, RB, NF, EPI, NE><<<grid, kThreads, 0, s>>>(in, zmask, adv, dv, g.rows, tw, twrc, advB, em);
  REG_LAUNCH();
}

template <typename T, int NF, int EPI, int NE = 0>
void c2r(const Grid& g, cudaStream_t s, const RowsSpec<T, NF>& in, int zmask, const AdvEpi<T>& adv,
         const DivEpi<T>& dv, double bytes, const cx<T>* tw, const cx<T>* twrc,
         const AdvEpi<T>& advB = AdvEpi<T>{}, const Emit<T>& em = Emit<T>{}) {
  switch (g.L) {
    case 8: return c2r_L<T, 8, NF, EPI, NE>(g, s, in, zmask, adv, dv, bytes, tw, twrc, advB, em);
    case 16: return c2r_L<T, 16, NF, EPI, NE>(g, s, in, zmask, adv, dv, bytes, tw, twrc, advB, em);
    case 32: return c2r_L<T, 32, NF, EPI, NE>(g, s, in, zmask, adv, dv, bytes, tw, twrc, advB, em);
    case 64: return c2r_L<T, 64, NF, EPI, NE>(g, s, in, zmask, adv, dv, bytes, tw, twrc, advB, em);
    case 128: return c2r_L<T, 128, NF, EPI, NE>(g, s, in, zmask, adv, dv, bytes, tw, twrc, advB, em);
    case 256: return c2r_L<T, 256, NF, EPI, NE>(g, s, in, zmask, adv, dv, bytes, tw, twrc, advB, em);
    case 512: return c2r_L<T, 512, NF, EPI, NE>(g, s, in, zmask, adv, dv, bytes, tw, twrc, advB, em);
  }
  throw StatusError{1, "unsupported last-axis length"};
}

template <typename T, int L, int TC>
void deriv_launch(const cx<T>* in, cx<T>* out, const cx<T>* add, long s, long outer, const cx<T>* tw,
                  cudaStream_t st) {
  ProfScope ps(KK_COLS, st, (double)s * outer * L * sizeof(cx<T>) * (add ? 3.0 : 2.0),
               (double)s * outer * (2.0 * fft_flops<L>() + L * (add ? 4.0 : 2.0)));
  dim3 grid((unsigned)(s / TC), (unsigned)outer);
  k_cols_deriv<T, L, TC><<<grid, kThreads, 0, st>>>(in, out, add, s, tw);
  REG_LAUNCH();
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library)
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
inline EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      (void)cudaGetLastError();
      p = nullptr;
    }
    return reinterpret_cast<EncodeTiledFn>(p);
  }();
  return fn;
}

// Tensor map of the strided pencils of one column pass (rows of s complex
// values as 4-byte elements, outer * L rows; box TC complex x L rows). False
// when the shape is not expressible (L > 256 rows per box) or the encoder
// refuses it.
template <typename T, int L, int TC>
bool cols_tensor_map(CUtensorMap* m, const cx<T>* in, long s, long outer) {
  if (L > 256) return false;
  EncodeTiledFn fn = encode_tiled();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)s * sizeof(cx<T>) / 4, (cuuint64_t)outer * L};
  cuuint64_t strides[1] = {(cuuint64_t)s * sizeof(cx<T>)};
  cuuint32_t box[2] = {(cuuint32_t)(TC * sizeof(cx<T>) / 4), (cuuint32_t)L};
  cuuint32_t es[2] = {1, 1};
  if (((uintptr_t)in & 15) || (strides[0] & 15) || box[0] > 256) return false;
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<cx<T>*>(in), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}


// variant 0: persistent double-buffered, tile width TCmax (tiles by TMA where
// a tensor map can describe them, else by cp.async); variants 1..3:
// one block per tile with widths TCmax, TCmax/2, 4
template <typename T, int L, int TC, bool PERSIST>
void deriv2_launch(const cx<T>* in, cx<T>* out, const cx<T>* add, long s, long outer, const cx<T>* tw,
                   cudaStream_t st) {
  constexpr int R0 = Plan<L>::R[0], R1 = Plan<L>::R[1];
  constexpr int NT = TC * (R0 > L / R0 ? R0 : L / R0);
  ProfScope ps(KK_COLS, st, (double)s * outer * L * sizeof(cx<T>) * (add ? 3.0 : 2.0),
               (double)s * outer * (2.0 * fft_flops<L>() + L * (add ? 4.0 : 2.0)));
  const long ntx = s / TC, ntiles = ntx * outer;
  if constexpr (PERSIST) {
    constexpr size_t smem = 2 * (size_t)L * TC * sizeof(cx<T>);
    CUtensorMap map;
    if (cols_tensor_map<T, L, TC>(&map, in, s, outer)) {
      // resident blocks of one wave, computed once per instantiation (thread-safe static initialisation;
      // retried on the next call if a query throws)
      static const int resident_t = persistent_wave(k_cols_deriv2t<T, L, TC, R0, R1>, NT, smem);
      long grid = ntiles < resident_t ? ntiles : resident_t;
      k_cols_deriv2t<T, L, TC, R0, R1><<<(unsigned)grid, NT, smem, st>>>(map, out, add, s, (int)ntx, (int)ntiles, tw);
      REG_LAUNCH();
      return;
    }
    static const int resident = persistent_wave(k_cols_deriv2p<T, L, TC, R0, R1>, NT, smem);
    long grid = ntiles < resident ? ntiles : resident;
    k_cols_deriv2p<T, L, TC, R0, R1><<<(unsigned)grid, NT, smem, st>>>(in, out, add, s, (int)ntx, (int)ntiles, tw);
  } else {
    dim3 grid((unsigned)(s / TC), (unsigned)outer);
    k_cols_deriv2<T, L, TC, R0, R1><<<grid, NT, 0, st>>>(in, out, add, s, tw);
  }
  REG_LAUNCH();
}

template <typename T, int L>
constexpr int tc_max() {
  constexpr int TCmax0 = sizeof(T) == 4 ? 16 : 8;
  return (L * TCmax0 * sizeof(cx<T>) > 32768) ? TCmax0 / 2 : TCmax0;
}

template <typename T, int L>
bool deriv2_variant_ok(int v, long s, long outer) {
  constexpr int TM = tc_max<T, L>();
  const int tc[4] = {TM, TM, TM / 2 >= 2 ? TM / 2 : 2, 4};
  if (s < tc[v] || s % tc[v]) return false;
  if (v == 0) return (s / TM) * outer >= 2 * 152;  // persistent form only for large grids
  return true;
}

template <typename T, int L>
void deriv2_variant(int v, const cx<T>* in, cx<T>* out, const cx<T>* add, long s, long outer, const cx<T>* tw,
                    cudaStream_t st) {
  constexpr int TM = tc_max<T, L>();
  switch (v) {
    case 0: return deriv2_launch<T, L, TM, true>(in, out, add, s, outer, tw, st);
    case 1: return deriv2_launch<T, L, TM, false>(in, out, add, s, outer, tw, st);
    case 2: return deriv2_launch<T, L, (TM / 2 >= 2 ? TM / 2 : 2), false>(in, out, add, s, outer, tw, st);
    default: return deriv2_launch<T, L, 4, false>(in, out, add, s, outer, tw, st);
  }
}

// Autotuner of the column derivative pass (choices also persisted, see
// tune.cu). Fields larger than 16 MB stream
// through DRAM (the input was written by the previous pass, partly still in
// L2): there the persistent double-buffered variant is used whenever it is
// admissible; isolated trials, warm or flushed, do not reproduce that state
// and ranked the variants wrongly. Smaller fields live in L2 in use; on the
// first use of such a (precision, length, stride, batch) shape every
// admissible variant runs three times on scratch memory, timed with CUDA
// events on the calling stream, and the fastest is kept for the process.
// REG_AUTOTUNE=0 skips the trials (the first admissible variant in the order
// 0..3 is used).
struct Tuner {
  std::mutex mu;
  std::map<std::tuple<int, int, long, long>, int> best;
  void* scratch = nullptr;
  size_t scratch_bytes = 0;
};
inline Tuner& tuner() {
  static Tuner t;
  return t;
}

template <typename T, int L>
int deriv2_choice(long s, long outer, const cx<T>* tw, cudaStream_t st) {
  Tuner& tu = tuner();
  std::lock_guard<std::mutex> lk(tu.mu);
  auto key = std::make_tuple((int)sizeof(T), L, s, outer);
  auto it = tu.best.find(key);
  if (it != tu.best.end()) return it->second;
  const std::string pkey = tune_device_tag() + "|cols|" + (sizeof(T) == 4 ? "f32" : "f64") + "|L" +
                           std::to_string(L) + "|s" + std::to_string(s) + "|outer" + std::to_string(outer);
  int pick = tune_lookup(pkey);
  if (pick >= 0 && pick < 4 && deriv2_variant_ok<T, L>(pick, s, outer)) {
    tu.best[key] = pick;
    return pick;
  }
  pick = -1;
  const char* env = getenv("REG_AUTOTUNE");
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  REG_CUDA(cudaStreamIsCapturing(st, &cs));
  bool tune = !(env && env[0] == '0') && cs == cudaStreamCaptureStatusNone;  // no trials inside a capture
  const size_t field = (size_t)s * outer * L * sizeof(cx<T>);
  if (field > (16ull << 20) && deriv2_variant_ok<T, L>(0, s, outer)) {
    tu.best[key] = 0;
    return 0;
  }
  if (tune && 2 * field > tu.scratch_bytes) {
    if (tu.scratch) cudaFree(tu.scratch);
    tu.scratch = nullptr;
    tu.scratch_bytes = 0;
    if (cudaMalloc(&tu.scratch, 2 * field) != cudaSuccess) {
      (void)cudaGetLastError();
      tune = false;
    } else {
      tu.scratch_bytes = 2 * field;
    }
  }
  if (tune) {
    cx<T>* a = (cx<T>*)tu.scratch;
    cx<T>* b = a + s * outer * L;
    REG_CUDA(cudaMemsetAsync(a, 0, field, st));
    cudaEvent_t e0, e1;
    REG_CUDA(cudaEventCreate(&e0));
    REG_CUDA(cudaEventCreate(&e1));
    float bestms = 1e30f;
    for (int v = 0; v < 4; ++v) {
      if (!deriv2_variant_ok<T, L>(v, s, outer)) continue;
      deriv2_variant<T, L>(v, a, b, nullptr, s, outer, tw, st);  // first run (lazy set-up)
      float total = 0;
      for (int r = 0; r < 3; ++r) {
        REG_CUDA(cudaEventRecord(e0, st));
        deriv2_variant<T, L>(v, a, b, nullptr, s, outer, tw, st);
        REG_CUDA(cudaEventRecord(e1, st));
        REG_CUDA(cudaEventSynchronize(e1));
        float ms = 0;
        REG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        total += ms;
      }
      if (total < bestms) {
        bestms = total;
        pick = v;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }
  for (int v = 0; v < 4 && pick < 0; ++v)
    if (deriv2_variant_ok<T, L>(v, s, outer)) pick = v;
  tu.best[key] = pick;
  if (pick >= 0) tune_store(pkey, pick);
  return pick;
}

template <typename T, int L>
void deriv_tc(const cx<T>* in, cx<T>* out, const cx<T>* add, long s, long outer, const cx<T>* tw, cudaStream_t st) {
  constexpr int TCmax = tc_max<T, L>();
  if constexpr (Plan<L>::S == 2) {
    // two-stage plans keep the column in registers between the stages
    int v = deriv2_choice<T, L>(s, outer, tw, st);
    if (v >= 0) return deriv2_variant<T, L>(v, in, out, add, s, outer, tw, st);
  }
  if (s >= TCmax) return deriv_launch<T, L, TCmax>(in, out, add, s, outer, tw, st);
  if (s >= 4) return deriv_launch<T, L, 4>(in, out, add, s, outer, tw, st);
  return deriv_launch<T, L, 2>(in, out, add, s, outer, tw, st);
}

// derivative along strided axis `axis` of the z-spectral rows
template <typename T>
void deriv(const Grid& g, const Spectral<T>& sp, int axis, const cx<T>* in, cx<T>* out, const cx<T>* add,
           cudaStream_t st) {
  long s = g.M;
  for (int a = axis + 1; a < g.d - 1; ++a) s *= g.n[a];
  long outer = g.Nc / (s * g.n[axis]);
  const cx<T>* tw = sp.twiddles(g.n[axis]);
  switch (g.n[axis]) {
    case 8: return deriv_tc<T, 8>(in, out, add, s, outer, tw, st);
    case 16: return deriv_tc<T, 16>(in, out, add, s, outer, tw, st);
    case 32: return deriv_tc<T, 32>(in, out, add, s, outer, tw, st);
    case 64: return deriv_tc<T, 64>(in, out, add, s, outer, tw, st);
    case 128: return deriv_tc<T, 128>(in, out, add, s, outer, tw, st);
    case 256: return deriv_tc<T, 256>(in, out, add, s, outer, tw, st);
    case 512: return deriv_tc<T, 512>(in, out, add, s, outer, tw, st);
  }
  throw StatusError{1, "unsupported axis length"};
}

// pencil geometry of a strided pass along `axis` of the z-spectral rows:
// element j of pencil (outer, inner) at outer*n*s + j*s + inner
inline void col_geometry(const Grid& g, int axis, long* s, long* outer) {
  long st = g.M;
  for (int a = axis + 1; a < g.d - 1; ++a) st *= g.n[a];
  *s = st;
  *outer = g.Nc / (st * g.n[axis]);
}

// One strided derivative pass of a stage: out = D_axis in (+ add)
template <typename T>
struct ColJob {
  int axis;
  const cx<T>* in;
  cx<T>* out;
  const cx<T>* add;
  int rev = 0;  // walk the tiles from the last one
};

template <int L>
void cols_pairs_L(const Spectral<float>& sp, const Grid& g, const ColJob<float>* jobs, int nj, cudaStream_t st) {
  constexpr int R0 = Plan<L>::R[0], R1 = Plan<L>::R[1];
  constexpr int NT = 8 * (L / R0 > R0 ? L / R0 : R0);
  constexpr size_t smem = 2 * (size_t)L * 16 * sizeof(float2);
  CUtensorMap maps[kColJobs];
  ColJobs J{};
  J.nj = nj;
  double bytes = 0, flops = 0;
  int acc = 0;
  for (int q = 0; q < nj; ++q) {
    long s, outer;
    col_geometry(g, jobs[q].axis, &s, &outer);
    if (!cols_tensor_map<float, L, 16>(&maps[q], jobs[q].in, s, outer))
      throw StatusError{3, "column pass: tensor map rejected"};
    J.out[q] = jobs[q].out;
    J.add[q] = jobs[q].add;
    J.rev[q] = jobs[q].rev;
    J.s[q] = s;
    J.ntx[q] = (int)(s / 16);
    J.start[q] = acc;
    acc += (int)(s / 16 * outer);
    bytes += (double)s * outer * L * sizeof(float2) * (jobs[q].add ? 3.0 : 2.0);
    flops += (double)s * outer * (2.0 * fft_flops<L>() + L * (jobs[q].add ? 4.0 : 2.0));
  }
  for (int q = nj; q < kColJobs; ++q) maps[q] = maps[0];
  J.start[nj] = acc;
  ProfScope ps(KK_COLS, st, bytes, flops);
  // resident blocks of one wave, computed once (thread-safe static initialisation)
  static const int resident = persistent_wave(k_cols_pairs<L, R0, R1>, NT, smem);
  const int grid = acc < resident ? acc : resident;
  k_cols_pairs<L, R0, R1><<<grid, NT, smem, st>>>(maps[0], maps[1], maps[2], maps[3], J, sp.pair_twiddles(L));
  REG_LAUNCH();
}

// The strided passes of one stage in as few launches as possible: with single
// precision, two-stage radix plans and fields that stream through DRAM (the
// persistent regime, more than 16 MB per field), all jobs of one axis length
// share one launch of k_cols_pairs. Returns false without launching anything
// when some job does not qualify; the caller then runs deriv() per job.
template <typename T>
bool cols_pairs(const Spectral<T>& sp, const ColJob<T>* jobs, int nj, cudaStream_t st) {
  if constexpr (sizeof(T) != 4) {
    return false;
  } else {
    const Grid& g = sp.grid();
    const char* env = getenv("REG_PAIRED_COLS");
    if (env && env[0] == '0') return false;
    for (int q = 0; q < nj; ++q) {
      const int L = g.n[jobs[q].axis];
      long s, outer;
      col_geometry(g, jobs[q].axis, &s, &outer);
      if (L < 32 || L > 256 || s % 16 || (size_t)s * outer * L * sizeof(float2) <= (16ull << 20) ||
          ((uintptr_t)jobs[q].in & 15) || ((uintptr_t)jobs[q].out & 15) || ((uintptr_t)jobs[q].add & 15) ||
          !sp.pair_twiddles(L))
        return false;
    }
    // The axis-1 passes run first and walk their tiles from the last one: their
    // last tiles (largest outer index) read the rows the preceding row pass
    // wrote last, still in L2. Measured on the 256^3 matvec: 224.8 -> 222.3 ms
    // against the given order; reversing the axis-0 passes as well changed nothing.
    ColJob<T> ord[kColJobs];
    {
      int m = 0;
      for (int q = 0; q < nj; ++q)
        if (jobs[q].axis == 1) {
          ord[m] = jobs[q];
          ord[m++].rev = 1;
        }
      for (int q = 0; q < nj; ++q)
        if (jobs[q].axis != 1) ord[m++] = jobs[q];
      jobs = ord;
    }
    // one launch per distinct axis length, jobs in that order
    for (int done = 0; done < nj;) {
      const int L = g.n[jobs[done].axis];
      ColJob<float> grp[kColJobs];
      int m = 0;
      for (int q = done; q < nj && g.n[jobs[q].axis] == L; ++q) grp[m++] = jobs[q];
      switch (L) {
        case 32: cols_pairs_L<32>(sp, g, grp, m, st); break;
        case 64: cols_pairs_L<64>(sp, g, grp, m, st); break;
        case 128: cols_pairs_L<128>(sp, g, grp, m, st); break;
        default: cols_pairs_L<256>(sp, g, grp, m, st); break;
      }
      done += m;
    }
    return true;
  }
}

// One advection stage on u. u_ready: U already holds the packed spectrum of u
// (emitted by the previous stage's row pass), so no real-to-complex pass
// runs. emit: the row pass leaves the spectrum of its out1 values in U for
// the next stage.
template <typename T>
void adv_stage_impl(Spectral<T>& sp, const T* u, const AdvEpi<T>& e, cx<T>* U, cx<T>* Zx, cx<T>* Zy, bool u_ready,
                    bool emit) {
  const Grid& g = sp.grid();
  cudaStream_t s = sp.stream();
  const cx<T>* tw = sp.twiddles(g.M);
  const cx<T>* twrc = sp.rc_twiddles();
  if (!u_ready) {
    RowsIn<T, 1> in1{{u}};
    RowsOut<T, 1> out1{{U}};
    r2c<T, 1, false>(g, s, in1, nullptr, out1, 0, tw, twrc);
  }
  const int d = g.d;
  double bytes = (double)g.N * sizeof(T) *
                 (d + (e.G[0] ? d : 0) + (e.Sout ? d + 1 : 0) +
                  (e.out1 ? d + (e.src ? 1 : (e.gm[0] ? 2 * d : 0)) + (e.y ? 1 : 0) + (e.stage == 1 ? 2 : 1) -
                                (e.out1_spectral_only ? 1 : 0)
                          : 0) +
                  (emit ? 1 : 0));
  DivEpi<T> none{};
  Emit<T> em{};
  em.out[0] = U;
  if (d == 3) {
    const ColJob<T> jobs[2] = {{0, U, Zx, nullptr}, {1, U, Zy, nullptr}};
    if (!cols_pairs<T>(sp, jobs, 2, s)) {
      // the two strided passes are independent: the x pass runs on the second
      // stream, so each fills the other's last partial wave of blocks
      cudaStream_t s2 = sp.aux_stream();
      REG_CUDA(cudaEventRecord(sp.fork_event(), s));
      REG_CUDA(cudaStreamWaitEvent(s2, sp.fork_event(), 0));
      deriv<T>(g, sp, 0, U, Zx, nullptr, s2);
      deriv<T>(g, sp, 1, U, Zy, nullptr, s);
      REG_CUDA(cudaEventRecord(sp.join_event(), s2));
      REG_CUDA(cudaStreamWaitEvent(s, sp.join_event(), 0));
    }
    RowsSpec<T, 3> in{{Zx, Zy, U}};
    if (emit) c2r<T, 3, EPI_ADV, 1>(g, s, in, 1 << 2, e, none, bytes, tw, twrc, AdvEpi<T>{}, em);
    else c2r<T, 3, EPI_ADV>(g, s, in, 1 << 2, e, none, bytes, tw, twrc);
  } else {
    deriv<T>(g, sp, 0, U, Zy, nullptr, s);
    RowsSpec<T, 2> in{{Zy, U}};
    if (emit) c2r<T, 2, EPI_ADV, 1>(g, s, in, 1 << 1, e, none, bytes, tw, twrc, AdvEpi<T>{}, em);
    else c2r<T, 2, EPI_ADV>(g, s, in, 1 << 1, e, none, bytes, tw, twrc);
  }
}

// Two advection stages of 3D fields uA and uB in one pass sequence: one
// real-to-complex pass over both, the four strided passes, one
// complex-to-real pass of six spectra with both epilogues.
template <typename T>
void adv2_stage_impl(Spectral<T>& sp, const T* uA, const AdvEpi<T>& eA, const T* uB, const AdvEpi<T>& eB,
                     cx<T>* const* Z) {
  const Grid& g = sp.grid();
  cudaStream_t s = sp.stream();
  const cx<T>* tw = sp.twiddles(g.M);
  const cx<T>* twrc = sp.rc_twiddles();
  cx<T>* UA = Z[0];
  cx<T>* XA = Z[1];
  cx<T>* YA = Z[2];
  cx<T>* UB = Z[3];
  cx<T>* XB = Z[4];
  cx<T>* YB = Z[5];
  RowsIn<T, 2> in2{{uA, uB}};
  RowsOut<T, 2> out2{{UA, UB}};
  r2c<T, 2, false>(g, s, in2, nullptr, out2, 0, tw, twrc);
  auto epi_bytes = [&](const AdvEpi<T>& e) {
    return (double)g.N * sizeof(T) *
           (3 + (e.G[0] ? 3 : 0) + (e.Sout ? 3 + 1 : 0) +
            (e.out1 ? 3 + ((e.src || e.src_from_a) ? (e.src ? 1 : 0) : (e.gm[0] ? 6 : 0)) + (e.y ? 1 : 0) +
                          (e.stage == 1 ? 2 : 1)
                    : 0));
  };
  const ColJob<T> jobs[4] = {{0, UA, XA, nullptr}, {0, UB, XB, nullptr}, {1, UA, YA, nullptr}, {1, UB, YB, nullptr}};
  if (!cols_pairs<T>(sp, jobs, 4, s)) {
    cudaStream_t s2 = sp.aux_stream();
    REG_CUDA(cudaEventRecord(sp.fork_event(), s));
    REG_CUDA(cudaStreamWaitEvent(s2, sp.fork_event(), 0));
    deriv<T>(g, sp, 0, UA, XA, nullptr, s2);
    deriv<T>(g, sp, 0, UB, XB, nullptr, s2);
    deriv<T>(g, sp, 1, UA, YA, nullptr, s);
    deriv<T>(g, sp, 1, UB, YB, nullptr, s);
    REG_CUDA(cudaEventRecord(sp.join_event(), s2));
    REG_CUDA(cudaStreamWaitEvent(s, sp.join_event(), 0));
  }
  DivEpi<T> none{};
  RowsSpec<T, 6> in6{{XA, YA, UA, XB, YB, UB}};
  // a velocity read by both epilogues (the same node, or n_c = 1) is counted once
  const bool shared_a = eA.out1 && eB.out1 && eA.a[0] == eB.a[0] && eA.a[1] == eB.a[1] && eA.a[2] == eB.a[2];
  const double bytes = epi_bytes(eA) + epi_bytes(eB) - (shared_a ? 3.0 * g.N * sizeof(T) : 0.0);
  AdvEpi<T> eB2 = eB;  // the second epilogue takes the first one's velocity values
  eB2.a_from_a = shared_a ? 1 : 0;
  c2r<T, 6, EPI_ADV2>(g, s, in6, (1 << 2) | (1 << 5), eA, none, bytes, tw, twrc, eB2);
}

template <typename T>
void div_stage_impl(Spectral<T>& sp, const T* lam, const T* a, const DivEpi<T>& e, cx<T>* Q0, cx<T>* Q1,
                    cx<T>* Q2) {
  const Grid& g = sp.grid();
  cudaStream_t s = sp.stream();
  const cx<T>* tw = sp.twiddles(g.M);
  const cx<T>* twrc = sp.rc_twiddles();
  const long N = g.N;
  AdvEpi<T> none{};
  double bytes = (double)N * sizeof(T) * (1 + (e.stage ? 1 : 0) + (e.stage == 1 ? 2 : 1) + (e.src ? 1 : 0));
  if (e.f_hi)
    bytes += (double)N * sizeof(T) *
             (g.d * (e.gmB ? 2 : 1) + (e.gmC ? g.d + 1 : 0) + 2.0 * e.nc * g.d * (e.f_lo ? 2 : 1));
  if (g.d == 3) {
    RowsIn<T, 3> in{{a, a + N, a + 2 * N}};
    RowsOut<T, 3> out{{Q0, Q1, Q2}};
    r2c<T, 3, true>(g, s, in, lam, out, 1 << 2, tw, twrc);
    // the two strided derivatives in place, independent of each other (one
    // launch); the row pass adds the three spectra on load
    const ColJob<T> jobs[2] = {{0, Q0, Q0, nullptr}, {1, Q1, Q1, nullptr}};
    if (cols_pairs<T>(sp, jobs, 2, s)) {
      RowsSpec<T, 3> sp3{{Q0, Q1, Q2}};
      c2r<T, 3, EPI_DIVS>(g, s, sp3, 0, none, e, bytes + 2.0 * N * sizeof(T), tw, twrc);
    } else {
      deriv<T>(g, sp, 1, Q1, Q2, Q2, s);
      deriv<T>(g, sp, 0, Q0, Q2, Q2, s);
      RowsSpec<T, 1> sp1{{Q2}};
      c2r<T, 1, EPI_DIV>(g, s, sp1, 0, none, e, bytes, tw, twrc);
    }
  } else {
    RowsIn<T, 2> in{{a, a + N}};
    RowsOut<T, 2> out{{Q0, Q1}};
    r2c<T, 2, true>(g, s, in, lam, out, 1 << 1, tw, twrc);
    deriv<T>(g, sp, 0, Q0, Q1, Q1, s);
    RowsSpec<T, 1> sp1{{Q1}};
    c2r<T, 1, EPI_DIV>(g, s, sp1, 0, none, e, bytes, tw, twrc);
  }
}

}  // namespace fused
}  // namespace reg
