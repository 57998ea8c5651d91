// C ABI of the coupled lattice-Boltzmann ice-crystal step (include/lbmice.h): parameter
// derivation, device state, kernel launches and CUDA-graph replay of step chunks.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <new>
#include <type_traits>
#include <utility>
#include <vector>

#include "../../include/lbmice.h"
#include "lbmice_adjoint.cuh"
#include "lbmice_aux.cuh"
#include "lbmice_step.cuh"

using namespace lbmice;

namespace {

constexpr double kA2 = 0.6267;   // Sec. 2.1: a2 of the sharp-interface mapping
constexpr double kHdrag = 2.757; // Sec. 2.2.1: drag constant h
constexpr int kTX = 32, kTY = 8; // destination tile of the step kernel
// Steps per captured graph: a multiple of 6, so the population double buffer (period 2) and
// the phi triple buffer (period 3) are back in their slots after each replay.
constexpr int kGraphSteps = 60;
constexpr int kStatBlocks = 608; // 4 x 152 SMs
constexpr int kPhases = 6;       // buffer rotation period: populations 2, phi planes 3
constexpr int kMapsPerPhase = 6; // tensor maps of one step's inputs (StepPtrs::tm)

}  // namespace

struct lbmice_ctx {
  lbmice_params p;
  Consts C;
  double Dphi3, lambda;
  int device = 0;
  cudaStream_t stream = nullptr;   // caller's stream: every launch goes here
  cudaStream_t capture = nullptr;  // private stream used only to record graphs
  int nplanes = 0;
  size_t elem = 4;                 // bytes per stored population
  void* pops[2] = {nullptr, nullptr};
  float* phi[3] = {nullptr, nullptr, nullptr};
  float* Um[2] = {nullptr, nullptr};   // 16-bit storage: U (zeroth moment of g), ping-pong
  float* rhom[2] = {nullptr, nullptr}; // 16-bit storage with flow: rho, ping-pong
  float* fieldbuf = nullptr;       // one contiguous float field, for host exports
  double* stat_partial = nullptr;
  double* stat_out = nullptr;
  double* stat_host = nullptr;     // pinned
  double* tip_dev = nullptr;       // (cos, sin) of up to LBMICE_MAX_RAYS rays, then their radii
  double* tip_host = nullptr;      // pinned, the same layout
  cudaGraphExec_t graph = nullptr;
  int64_t step = 0;
  // tensor maps of the march's L2 prefetch, kMapsPerPhase per step phase (step mod 6), in
  // device memory
  CUtensorMap* tmaps = nullptr;
};

namespace {

inline dim3 node_grid(const Consts& C, dim3 blk) {
  return dim3((C.nx + blk.x - 1) / blk.x, (C.ny + blk.y - 1) / blk.y);
}

// name of the last CUDA error this thread turned into an error code (lbmice_last_error)
thread_local const char* g_last_cuda_error = "none";

int cuda_err(cudaError_t e) {
  if (e == cudaSuccess) return LBMICE_OK;
  g_last_cuda_error = cudaGetErrorName(e);
  return e == cudaErrorMemoryAllocation ? LBMICE_ENOMEM : LBMICE_ECUDA;
}

#define LB_TRY(expr)                          \
  do {                                        \
    int rc_ = cuda_err(expr);                 \
    if (rc_ != LBMICE_OK) return rc_;         \
  } while (0)

int validate(const lbmice_params& p) {
  if (p.nx < 4 || p.ny < 4) return LBMICE_EINVAL;
  const long long pitch = ((long long)p.nx + 31) / 32 * 32;
  if (pitch * p.ny >= (1LL << 31)) return LBMICE_EINVAL;
  if (!(p.dx > 0) || !(p.dt > 0) || !(p.W0 > 0) || !(p.tau0 > 0)) return LBMICE_EINVAL;
  if (!(p.D >= 0) || !(p.eps >= 0 && p.eps < 1) || !(p.kappa_N >= 0)) return LBMICE_EINVAL;
  if (!std::isfinite(p.L_sat) || !std::isfinite(p.U_in) || !std::isfinite(p.lambda))
    return LBMICE_EINVAL;
  for (int f = 0; f < 4; ++f)
    if (p.bc[f] < LBMICE_BC_PERIODIC || p.bc[f] > LBMICE_BC_FREESLIP) return LBMICE_EINVAL;
  if ((p.bc[0] == LBMICE_BC_PERIODIC) != (p.bc[1] == LBMICE_BC_PERIODIC)) return LBMICE_EINVAL;
  if ((p.bc[2] == LBMICE_BC_PERIODIC) != (p.bc[3] == LBMICE_BC_PERIODIC)) return LBMICE_EINVAL;
  if (p.flow != 0 && p.flow != 1) return LBMICE_EINVAL;
  if (p.check_every < 0) return LBMICE_EINVAL;
  if (p.storage < LBMICE_STORAGE_F32 || p.storage > LBMICE_STORAGE_BF16) return LBMICE_EINVAL;
  if (p.stencil != 0 && p.stencil != 2 && p.stencil != 4 && p.stencil != 6 && p.stencil != 8)
    return LBMICE_EINVAL;
  if (p.fold != 0 && p.fold != 4 && p.fold != 6) return LBMICE_EINVAL;
  if (!std::isfinite(p.u_in) || std::fabs(p.u_in) >= std::sqrt(1.0 / 3.0)) return LBMICE_EUNSTABLE;
  if (p.flow && !(p.nu > 0)) return LBMICE_EUNSTABLE;  // tau_f = 3 nu + 1/2 must exceed 1/2
  return LBMICE_OK;
}

void derive(lbmice_t* h) {
  const lbmice_params& p = h->p;
  Consts& C = h->C;
  std::memset(&C, 0, sizeof(C));
  C.nx = p.nx;
  C.ny = p.ny;
  C.pitch = (p.nx + 31) / 32 * 32;
  C.pstride = (long long)C.pitch * p.ny;  // plane-major: [plane][ny][pitch]
  C.rstride = C.pitch;
  for (int f = 0; f < 4; ++f) C.bc[f] = p.bc[f];
  C.stencil = p.stencil == 0 ? 4 : p.stencil;
  C.fold = p.fold == 0 ? 6 : p.fold;
  const double Dphi = (p.W0 * p.W0 / p.tau0) * p.dt / (p.dx * p.dx);
  h->Dphi3 = 3.0 * Dphi;
  h->lambda = p.lambda > 0 ? p.lambda : p.tau0 * p.D / (kA2 * p.W0 * p.W0);
  const double Wlat = p.W0 / p.dx;
  const double tau_f = p.nu * 3.0 + 0.5;
  C.Dphi3 = (float)h->Dphi3;
  C.dt_tau0 = (float)(p.dt / p.tau0);
  C.lambda = (float)h->lambda;
  C.Dlat3 = (float)(3.0 * p.D * p.dt / (p.dx * p.dx));
  C.half_Lsat = (float)(0.5 * p.L_sat);
  C.eps = (float)p.eps;
  C.kNkeps = (float)(p.kappa_N * C.fold * p.eps);
  C.kdrag = (float)(kHdrag * p.nu / (4.0 * Wlat * Wlat));
  C.inv_tau_f = (float)(1.0 / tau_f);
  C.guo = (float)(1.0 - 0.5 / tau_f);
  C.U_in = (float)p.U_in;
  const double nxs[4] = {1, -1, 0, 0}, nys[4] = {0, 0, 1, -1};
  for (int f = 0; f < 4; ++f) {
    C.uin_x[f] = (float)(p.u_in * nxs[f]);
    C.uin_y[f] = (float)(p.u_in * nys[f]);
  }
}

void release(lbmice_t* h) {
  if (h->graph) cudaGraphExecDestroy(h->graph);
  for (void* b : h->pops) if (b) cudaFree(b);
  for (float* b : h->phi) if (b) cudaFree(b);
  for (float* b : h->Um) if (b) cudaFree(b);
  for (float* b : h->rhom) if (b) cudaFree(b);
  if (h->fieldbuf) cudaFree(h->fieldbuf);
  if (h->stat_partial) cudaFree(h->stat_partial);
  if (h->stat_out) cudaFree(h->stat_out);
  if (h->stat_host) cudaFreeHost(h->stat_host);
  if (h->tip_dev) cudaFree(h->tip_dev);
  if (h->tip_host) cudaFreeHost(h->tip_host);
  if (h->tmaps) cudaFree(h->tmaps);
  if (h->capture) cudaStreamDestroy(h->capture);
  delete h;
}

// bytes of one population buffer: nplanes planes of ny rows of pitch values, whatever the
// interleaving of planes and rows
size_t pop_bytes(const lbmice_t* h) {
  return h->elem * (size_t)h->nplanes * (size_t)h->C.pitch * (size_t)h->C.ny;
}
size_t field_bytes(const lbmice_t* h) {
  return sizeof(float) * (size_t)h->C.pitch * (size_t)h->C.ny;
}
bool dev16(const lbmice_t* h) { return h->p.storage != LBMICE_STORAGE_F32; }

// cuTensorMapEncodeTiled of the driver, through the runtime's entry-point query (no link
// against the driver library).
PFN_cuTensorMapEncodeTiled_v12000 encode_tiled() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// A tiled tensor map of rank 2 or 3 over base: dims[0] the contiguous extent (elements),
// strides[i] the bytes between steps of dimension i + 1, box the box extents.
bool encode_map(CUtensorMap* m, CUtensorMapDataType t, int rank, const void* base,
                const uint64_t* dims, const uint64_t* strides, const uint32_t* box) {
  auto fn = encode_tiled();
  if (!fn) return false;
  cuuint64_t d[3], st[2];
  cuuint32_t b[3], es[3] = {1, 1, 1};
  for (int i = 0; i < rank; ++i) {
    d[i] = dims[i];
    b[i] = box[i];
  }
  for (int i = 0; i + 1 < rank; ++i) st[i] = strides[i];
  return fn(m, t, (cuuint32_t)rank, const_cast<void*>(base), d, st, b, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

// The maps of every step phase (the boxes of one march pass: 8 rows of a strip), encoded on
// the host and copied to the device once; the buffers never move.
int make_tensor_maps(lbmice_t* h) {
  // Every storage: phi^n in boxes of 8 rows x 40 columns, the march's phi ring blocks (slot
  // 5). The L2 prefetch boxes (slots 0..4) for 16-bit storage only: FP32 storage runs the
  // plain march, since prefetching its bandwidth-bound steps measured 15 B per node of
  // extra DRAM reads and no gain, while the issue-bound 16-bit steps gain 3%.
  std::vector<CUtensorMap> maps(kPhases * kMapsPerPhase);
  std::memset(maps.data(), 0, sizeof(CUtensorMap) * maps.size());
  const uint64_t P = h->C.pitch, NY = h->C.ny, Q = h->C.pstride;
  const uint32_t R = kMarchRows;
  bool ok = true;
  for (int ph = 0; ph < kPhases && ok; ++ph) {
    CUtensorMap* m = &maps[ph * kMapsPerPhase];
    const char* pin = static_cast<const char*>(h->pops[ph & 1]);
    const uint64_t d1[2] = {P, NY}, s1[1] = {P * 4};
    const uint32_t b1[2] = {36, R}, b5[2] = {kMarchPW, R};
    ok = ok && encode_map(&m[5], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, h->phi[ph % 3], d1, s1, b5);
    if (!dev16(h)) continue;
    const uint32_t L = h->p.flow ? 3 : 2;
    const uint64_t dv[3] = {8 * P, NY, L}, sv[2] = {16 * P, 18 * Q};
    const uint32_t bv[3] = {256, R, L};
    ok = ok && encode_map(&m[0], CU_TENSOR_MAP_DATA_TYPE_UINT16, 3, pin, dv, sv, bv);
    ok = ok && encode_map(&m[1], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, h->Um[ph & 1], d1, s1, b1);
    if (h->p.flow)
      ok = ok && encode_map(&m[2], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, h->rhom[ph & 1], d1, s1, b1);
    ok = ok && encode_map(&m[4], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, h->phi[(ph + 2) % 3], d1, s1, b1);
  }
  if (!ok) return LBMICE_ECUDA;
  LB_TRY(cudaMalloc(&h->tmaps, sizeof(CUtensorMap) * maps.size()));
  LB_TRY(cudaMemcpy(h->tmaps, maps.data(), sizeof(CUtensorMap) * maps.size(),
                    cudaMemcpyHostToDevice));
  return LBMICE_OK;
}

// Run f with a tag value of the handle's storage type.
template <class Fn>
int with_storage(const lbmice_t* h, Fn&& fn) {
  switch (h->p.storage) {
    case LBMICE_STORAGE_F16: return fn(F16{});
    case LBMICE_STORAGE_BF16: return fn(BF16{});
    default: return fn(F32{});
  }
}

// Segment height of the march for one grid on a device of sms SMs (4 CTAs per SM). Each
// segment collides two rows below its first in a prologue pass, and the last wave of CTAs
// may fill the GPU only in part; among heights of 40 .. 96 rows (multiples of the 8-row pass)
// that give at least one and a half waves, take the one that maximises
// (waves / waves begun) x H / (H + 2). A grid too small for any of them takes the tallest of
// 32, 16 rows that gives one and a half waves, else 8. (A batch, which has CTAs enough, walks
// every member in segments of 64.) At 2048 x 2048 on 152 SMs: 80 rows, 1794 CTAs, 2.95 waves.
int march_seg_rows(int nx, int ny, int sms) {
  const long long slots = 4LL * sms;
  const auto units = [&](int H) { return (long long)march_strips(nx) * ((ny + H - 1) / H); };
  int best = 0;
  double best_score = 0.0;
  for (int H = 40; H <= 96; H += kMarchRows) {
    const long long u = units(H);
    if (2 * u < 3 * slots) continue;
    const double waves = (double)u / (double)slots;
    const double score = waves / std::ceil(waves) * H / (H + 2.0);
    if (score > best_score) {
      best_score = score;
      best = H;
    }
  }
  if (best) return best;
  for (int H = 32; H > kMarchRows; H /= 2)
    if (2 * units(H) >= 3 * slots) return H;
  return kMarchRows;
}

// Launch grid of the march over one grid: one CTA per (strip, segment of H rows).
long long march_units(const Consts& C, int H) {
  return (long long)march_strips(C.nx) * ((C.ny + H - 1) / H);
}
dim3 march_grid(const Consts& C) {
  return dim3(march_strips(C.nx), (C.ny + C.seg_rows - 1) / C.seg_rows);
}

// Opt the march kernels of this storage into the shared memory they use (above 48 KB).
int march_attributes(const lbmice_t* h) {
  return with_storage(h, [&](auto tag) -> int {
    using S = decltype(tag);
    cudaError_t e = cudaSuccess;
    auto set = [&](auto kern, size_t bytes) {
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    };
    set(march_kernel<true, S, MARCH_PREFETCH>, march_smem_bytes<true>());
    set(march_kernel<false, S, MARCH_PREFETCH>, march_smem_bytes<false>());
    set(march_kernel<true, S, MARCH_PLAIN>, march_smem_bytes<true>());
    set(march_kernel<false, S, MARCH_PLAIN>, march_smem_bytes<false>());
    constexpr int M = Storage<S>::DEV ? MARCH_PREFETCH : MARCH_PLAIN;
    set(batch_march_kernel<true, S, M>, march_smem_bytes<true>());
    set(batch_march_kernel<false, S, M>, march_smem_bytes<false>());
    return cuda_err(e);
  });
}

// One step of grid h on the given buffers.
int launch_step_ptrs(const lbmice_t* h, const StepPtrs& P, cudaStream_t st) {
  if (h->C.stencil == 4 && h->C.fold == 6) {
    // the default scheme (E4, six-fold): the column march, its populations prefetched into
    // L2 by TMA when the step's buffers have tensor maps (16-bit storage)
    const dim3 grid = march_grid(h->C);
    return with_storage(h, [&](auto tag) {
      using S = decltype(tag);
      auto go = [&](auto flow, auto pref) {
        constexpr bool F = decltype(flow)::value;
        constexpr int M = decltype(pref)::value ? MARCH_PREFETCH : MARCH_PLAIN;
        march_kernel<F, S, M><<<grid, kMarchThreads, march_smem_bytes<F>(), st>>>(h->C, P);
      };
      const bool pref = dev16(h) && P.tm != nullptr;
      if (h->p.flow) {
        if (pref) go(std::true_type{}, std::true_type{}); else go(std::true_type{}, std::false_type{});
      } else {
        if (pref) go(std::false_type{}, std::true_type{}); else go(std::false_type{}, std::false_type{});
      }
      return cuda_err(cudaGetLastError());
    });
  }
  // every other stencil and fold: the 2D tile of radius 2 (E6 and E8 reach two nodes out:
  // phi halo 3)
  const dim3 grd((h->C.nx + kTX - 1) / kTX, (h->C.ny + kTY - 1) / kTY), blk(kTX * kTY);
  return with_storage(h, [&](auto tag) {
    using S = decltype(tag);
    if (h->p.flow)
      step_kernel<kTX, kTY, true, S, 2>
          <<<grd, blk, Tile<kTX, kTY, 2>::template smem_bytes<true>(), st>>>(h->C, P);
    else
      step_kernel<kTX, kTY, false, S, 2>
          <<<grd, blk, Tile<kTX, kTY, 2>::template smem_bytes<false>(), st>>>(h->C, P);
    return cuda_err(cudaGetLastError());
  });
}

StepPtrs step_ptrs(const lbmice_t* h, int ph);

// Step s of grid h on its own rotating buffers (phase s mod 6 of the buffer rotation).
int launch_step(lbmice_t* h, int64_t s, cudaStream_t st) {
  return launch_step_ptrs(h, step_ptrs(h, (int)(s % kPhases)), st);
}

int ensure_graph(lbmice_t* h) {
  if (h->graph) return LBMICE_OK;
  cudaGraph_t g = nullptr;
  LB_TRY(cudaStreamBeginCapture(h->capture, cudaStreamCaptureModeThreadLocal));
  int rc = LBMICE_OK;
  for (int s = 0; s < kGraphSteps && rc == LBMICE_OK; ++s) rc = launch_step(h, s, h->capture);
  cudaError_t e = cudaStreamEndCapture(h->capture, &g);
  if (rc != LBMICE_OK) { if (g) cudaGraphDestroy(g); return rc; }
  if (e != cudaSuccess) return cuda_err(e);
  e = cudaGraphInstantiate(&h->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) { h->graph = nullptr; return cuda_err(e); }
  return LBMICE_OK;
}

int run_stats(lbmice_t* h) {
  const int64_t s = h->step;
  int rc = with_storage(h, [&](auto tag) {
    using S = decltype(tag);
    stats_partial_kernel<S><<<kStatBlocks, kStatThreads, 0, h->stream>>>(
        h->C, h->p.flow, 0.5 * h->p.dx * h->p.dx, 0.5 * h->p.L_sat, h->pops[s & 1],
        h->phi[s % 3], h->phi[(s + 2) % 3], h->Um[s & 1], h->rhom[s & 1], h->stat_partial);
    return cuda_err(cudaGetLastError());
  });
  if (rc != LBMICE_OK) return rc;
  stats_final_kernel<<<1, 32, 0, h->stream>>>(h->stat_partial, kStatBlocks, h->stat_out);
  LB_TRY(cudaGetLastError());
  LB_TRY(cudaMemcpyAsync(h->stat_host, h->stat_out, kNStat * sizeof(double),
                         cudaMemcpyDeviceToHost, h->stream));
  LB_TRY(cudaStreamSynchronize(h->stream));
  // a bounded device-side wait (the march's phi-ring loads) that gave up since the last check
  unsigned int w = 0;
  LB_TRY(cudaMemcpyFromSymbol(&w, lbmice::wait_word, sizeof(w)));
  if (w) {
    const unsigned int z = 0;
    LB_TRY(cudaMemcpyToSymbol(lbmice::wait_word, &z, sizeof(z)));
    return LBMICE_ETIMEOUT;
  }
  return LBMICE_OK;
}

int equilibrium_from(lbmice_t* h, const double* phi, const double* U, const double* rho,
                     const double* ux, const double* uy) {
  if (!h->p.flow) ux = uy = rho = nullptr;  // fluid at rest: g^eq sees u = 0
  const dim3 blk(32, 8);
  const dim3 grd = node_grid(h->C, blk);
  const double eps = h->p.eps, kNkeps = h->p.kappa_N * h->C.fold * h->p.eps;
  int rc = with_storage(h, [&](auto tag) {
    using S = decltype(tag);
    if (h->p.flow)
      equilibrium_kernel<true, S><<<grd, blk, 0, h->stream>>>(
          h->C, h->Dphi3, eps, kNkeps, phi, U, rho, ux, uy, h->pops[0], h->phi[0], h->phi[2],
          h->Um[0], h->rhom[0]);
    else
      equilibrium_kernel<false, S><<<grd, blk, 0, h->stream>>>(
          h->C, h->Dphi3, eps, kNkeps, phi, U, rho, ux, uy, h->pops[0], h->phi[0], h->phi[2],
          h->Um[0], h->rhom[0]);
    return cuda_err(cudaGetLastError());
  });
  if (rc != LBMICE_OK) return rc;
  h->step = 0;
  return LBMICE_OK;
}

}  // namespace

extern "C" {

int lbmice_params_default(lbmice_params* p, int32_t nx, int32_t ny) {
  if (!p) return LBMICE_EINVAL;
  std::memset(p, 0, sizeof(*p));
  p->nx = nx;
  p->ny = ny;
  p->dx = 0.4;
  p->dt = 0.008;
  p->W0 = 1.0;
  p->tau0 = 1.0;
  p->D = 2.0;
  p->lambda = 0.0;
  p->L_sat = 1.0;
  p->eps = 0.05;
  p->kappa_N = 1.0;
  p->nu = 0.016;
  for (int f = 0; f < 4; ++f) p->bc[f] = LBMICE_BC_PERIODIC;
  p->stencil = 4;
  p->fold = 6;
  return LBMICE_OK;
}

int lbmice_create(const lbmice_params* p, void* stream, lbmice_t** out) {
  if (!out) return LBMICE_EINVAL;
  *out = nullptr;
  if (!p) return LBMICE_EINVAL;
  int rc = validate(*p);
  if (rc != LBMICE_OK) return rc;
  lbmice_t* h = new (std::nothrow) lbmice_ctx();
  if (!h) return LBMICE_ENOMEM;
  h->p = *p;
  derive(h);
  h->stream = static_cast<cudaStream_t>(stream);
  h->nplanes = p->flow ? 27 : 18;
  h->elem = p->storage == LBMICE_STORAGE_F32 ? 4 : 2;
  cudaError_t e = cudaGetDevice(&h->device);
  const size_t out_bytes = sizeof(float) * (size_t)p->nx * p->ny;
  const size_t phi_bytes = field_bytes(h);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->capture, cudaStreamNonBlocking);
  for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaMalloc(&h->pops[i], pop_bytes(h));
  for (int i = 0; i < 3 && e == cudaSuccess; ++i) e = cudaMalloc(&h->phi[i], phi_bytes);
  if (dev16(h)) {
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaMalloc(&h->Um[i], phi_bytes);
    for (int i = 0; i < 2 && e == cudaSuccess && p->flow; ++i)
      e = cudaMalloc(&h->rhom[i], phi_bytes);
  }
  if (e == cudaSuccess) e = cudaMalloc(&h->fieldbuf, out_bytes);
  if (e == cudaSuccess) e = cudaMalloc(&h->stat_partial, sizeof(double) * kStatBlocks * kNStat);
  if (e == cudaSuccess) e = cudaMalloc(&h->stat_out, sizeof(double) * 8);
  if (e == cudaSuccess) e = cudaMallocHost(&h->stat_host, sizeof(double) * 8);
  if (e == cudaSuccess) e = cudaMalloc(&h->tip_dev, sizeof(double) * 3 * LBMICE_MAX_RAYS);
  if (e == cudaSuccess) e = cudaMallocHost(&h->tip_host, sizeof(double) * 3 * LBMICE_MAX_RAYS);
  for (int i = 0; i < 2 && e == cudaSuccess; ++i)
    e = cudaMemsetAsync(h->pops[i], 0, pop_bytes(h), h->stream);
  for (int i = 0; i < 3 && e == cudaSuccess; ++i)
    e = cudaMemsetAsync(h->phi[i], 0, phi_bytes, h->stream);
  for (float* b : h->Um)
    if (b && e == cudaSuccess) e = cudaMemsetAsync(b, 0, phi_bytes, h->stream);
  for (float* b : h->rhom)
    if (b && e == cudaSuccess) e = cudaMemsetAsync(b, 0, phi_bytes, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    release(h);
    cudaGetLastError();  // clear a sticky-free error state left by a failed allocation
    return cuda_err(e);
  }
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess ||
      sms < 1)
    sms = 1;
  h->C.seg_rows = march_seg_rows(h->C.nx, h->C.ny, sms);
  rc = march_attributes(h);
  if (rc == LBMICE_OK) rc = make_tensor_maps(h);
  if (rc != LBMICE_OK) {
    release(h);
    cudaGetLastError();
    return rc;
  }
  *out = h;
  return LBMICE_OK;
}

int lbmice_init_seed(lbmice_t* h, double cx, double cy, double R0, double U0) {
  if (!h || !std::isfinite(cx) || !std::isfinite(cy) || !std::isfinite(R0) ||
      !std::isfinite(U0))
    return LBMICE_EINVAL;
  // The second population buffer is free before the first step: it holds the double seed
  // fields (phi and U, plus rho and u with flow: 16 or 40 bytes per node; it has at least 36
  // or 54).
  const size_t n = (size_t)h->p.nx * h->p.ny;
  double* f = reinterpret_cast<double*>(h->pops[1]);
  const bool fl = h->p.flow != 0;
  // velocity of the first inlet face along its inward normal (the fluid rests otherwise)
  double ux = 0.0, uy = 0.0;
  const double nxs[4] = {1, -1, 0, 0}, nys[4] = {0, 0, 1, -1};
  for (int face = 0; face < 4; ++face)
    if (h->p.flow && h->p.bc[face] == LBMICE_BC_INLET) {
      ux = h->p.u_in * nxs[face];
      uy = h->p.u_in * nys[face];
      break;
    }
  const dim3 blk(32, 8);
  const dim3 grd = node_grid(h->C, blk);
  double* rho = fl ? f + 2 * n : nullptr;
  double* uxf = fl ? f + 3 * n : nullptr;
  double* uyf = fl ? f + 4 * n : nullptr;
  seed_kernel<<<grd, blk, 0, h->stream>>>(h->p.nx, h->p.ny, cx, cy, R0, U0,
                                          std::sqrt(2.0) * h->p.W0 / h->p.dx, ux, uy, f,
                                          f + n, rho, uxf, uyf);
  LB_TRY(cudaGetLastError());
  return equilibrium_from(h, f, f + n, rho, uxf, uyf);
}

int lbmice_set_fields(lbmice_t* h, const double* phi, const double* U, const double* rho,
                      const double* ux, const double* uy, int32_t on_device) {
  if (!h || !phi || !U || (on_device != 0 && on_device != 1)) return LBMICE_EINVAL;
  if (on_device) return equilibrium_from(h, phi, U, rho, ux, uy);
  const size_t n = (size_t)h->p.nx * h->p.ny;
  double* f = reinterpret_cast<double*>(h->pops[1]);
  const bool fl = h->p.flow != 0;  // without flow the velocity inputs are ignored
  const double* src[5] = {phi, U, fl ? rho : nullptr, fl ? ux : nullptr, fl ? uy : nullptr};
  const double* dev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  for (int k = 0; k < 5; ++k) {
    if (!src[k]) continue;
    LB_TRY(cudaMemcpyAsync(f + k * n, src[k], n * sizeof(double), cudaMemcpyHostToDevice,
                           h->stream));
    dev[k] = f + k * n;
  }
  int rc = equilibrium_from(h, dev[0], dev[1], dev[2], dev[3], dev[4]);
  if (rc != LBMICE_OK) return rc;
  // pageable sources may be reused by the caller once this returns
  LB_TRY(cudaStreamSynchronize(h->stream));
  return LBMICE_OK;
}

int lbmice_step(lbmice_t* h, int64_t nsteps) {
  if (!h || nsteps < 0) return LBMICE_EINVAL;
  int64_t left = nsteps;
  const int64_t every = h->p.check_every;
  while (left > 0) {
    int64_t chunk = left;
    if (every > 0) chunk = std::min<int64_t>(left, every - (h->step % every));
    int64_t done = 0;
    while (done < chunk) {
      if (h->step % 6 == 0 && chunk - done >= kGraphSteps) {
        int rc = ensure_graph(h);
        if (rc != LBMICE_OK) return rc;
        LB_TRY(cudaGraphLaunch(h->graph, h->stream));
        h->step += kGraphSteps;
        done += kGraphSteps;
      } else {
        int rc = launch_step(h, h->step, h->stream);
        if (rc != LBMICE_OK) return rc;
        h->step += 1;
        done += 1;
      }
    }
    left -= chunk;
    if (every > 0 && h->step % every == 0) {
      int rc = run_stats(h);
      if (rc != LBMICE_OK) return rc;
      if (h->stat_host[4] != 0.0) return LBMICE_ENONFINITE;
    }
  }
  return LBMICE_OK;
}

}  // extern "C"

namespace {

// The pieces of the exact state, in blob order: populations, phi^n, phi^{n-1}, and with
// 16-bit storage U and rho of the current slot.
struct StatePart {
  void* ptr;
  size_t bytes;
};
int state_parts(lbmice_t* h, StatePart parts[5]) {
  const int64_t s = h->step;
  int n = 0;
  parts[n++] = {h->pops[s & 1], pop_bytes(h)};
  parts[n++] = {h->phi[s % 3], field_bytes(h)};
  parts[n++] = {h->phi[(s + 2) % 3], field_bytes(h)};
  if (h->Um[0]) parts[n++] = {h->Um[s & 1], field_bytes(h)};
  if (h->rhom[0]) parts[n++] = {h->rhom[s & 1], field_bytes(h)};
  return n;
}

}  // namespace

extern "C" size_t lbmice_state_bytes(const lbmice_t* h) {
  if (!h) return 0;
  StatePart parts[5];
  const int n = state_parts(const_cast<lbmice_t*>(h), parts);
  size_t total = 0;
  for (int k = 0; k < n; ++k) total += parts[k].bytes;
  return total;
}

namespace {

int copy_state(lbmice_t* h, void* blob, bool out, cudaMemcpyKind kind) {
  StatePart parts[5];
  const int n = state_parts(h, parts);
  char* b = static_cast<char*>(blob);
  for (int k = 0; k < n; ++k) {
    if (out)
      LB_TRY(cudaMemcpyAsync(b, parts[k].ptr, parts[k].bytes, kind, h->stream));
    else
      LB_TRY(cudaMemcpyAsync(parts[k].ptr, b, parts[k].bytes, kind, h->stream));
    b += parts[k].bytes;
  }
  return LBMICE_OK;
}

}  // namespace

extern "C" int lbmice_fields(lbmice_t* h, int32_t which, void* dst, size_t bytes,
                             int32_t dst_on_device) {
  if (!h || !dst || which < 0 || which > LBMICE_FIELD_STATE ||
      (dst_on_device != 0 && dst_on_device != 1))
    return LBMICE_EINVAL;
  const int64_t s = h->step;
  const size_t nx = h->p.nx, ny = h->p.ny;
  const cudaMemcpyKind kind = dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  const dim3 blk(32, 8);
  if (which == LBMICE_FIELD_STATE) {
    if (bytes < lbmice_state_bytes(h)) return LBMICE_EINVAL;
    int rc = copy_state(h, dst, true, kind);
    if (rc != LBMICE_OK) return rc;
  } else if (which == LBMICE_FIELD_POPS) {
    const size_t need = sizeof(float) * h->nplanes * nx * ny;
    if (bytes < need) return LBMICE_EINVAL;
    // decode one plane at a time (into dst directly, or through the field buffer)
    for (int q = 0; q < h->nplanes; ++q) {
      float* out = dst_on_device ? static_cast<float*>(dst) + (size_t)q * nx * ny
                                 : h->fieldbuf;
      int rc = with_storage(h, [&](auto tag) {
        using S = decltype(tag);
        decode_plane_kernel<S><<<node_grid(h->C, blk), blk, 0, h->stream>>>(
            h->C, h->pops[s & 1], q / 9, q % 9, h->phi[s % 3], h->Um[s & 1], h->rhom[s & 1],
            out);
        return cuda_err(cudaGetLastError());
      });
      if (rc != LBMICE_OK) return rc;
      if (!dst_on_device)
        LB_TRY(cudaMemcpyAsync(static_cast<float*>(dst) + (size_t)q * nx * ny, h->fieldbuf,
                               sizeof(float) * nx * ny, cudaMemcpyDeviceToHost, h->stream));
    }
  } else {
    const size_t need = sizeof(float) * nx * ny;
    if (bytes < need) return LBMICE_EINVAL;
    float* out = dst_on_device ? static_cast<float*>(dst) : h->fieldbuf;
    int rc = with_storage(h, [&](auto tag) {
      using S = decltype(tag);
      moment_kernel<S><<<node_grid(h->C, blk), blk, 0, h->stream>>>(
          h->C, which, h->p.flow, h->pops[s & 1], h->phi[s % 3], h->phi[(s + 2) % 3],
          h->Um[s & 1], h->rhom[s & 1], out);
      return cuda_err(cudaGetLastError());
    });
    if (rc != LBMICE_OK) return rc;
    if (!dst_on_device)
      LB_TRY(cudaMemcpyAsync(dst, h->fieldbuf, need, cudaMemcpyDeviceToHost, h->stream));
  }
  if (!dst_on_device) LB_TRY(cudaStreamSynchronize(h->stream));
  return LBMICE_OK;
}

extern "C" int lbmice_load(lbmice_t* h, int32_t which, const void* src, size_t bytes,
                           int32_t src_on_device) {
  if (!h || !src || (src_on_device != 0 && src_on_device != 1)) return LBMICE_EINVAL;
  if (which != LBMICE_FIELD_POPS && which != LBMICE_FIELD_PHI_PREV &&
      which != LBMICE_FIELD_STATE)
    return LBMICE_EINVAL;
  const int64_t s = h->step;
  const size_t nx = h->p.nx, ny = h->p.ny;
  const cudaMemcpyKind kind = src_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  const dim3 blk(32, 8);
  if (which == LBMICE_FIELD_STATE) {
    if (bytes < lbmice_state_bytes(h)) return LBMICE_EINVAL;
    int rc = copy_state(h, const_cast<void*>(src), false, kind);
    if (rc != LBMICE_OK) return rc;
  } else if (which == LBMICE_FIELD_POPS) {
    if (bytes < sizeof(float) * h->nplanes * nx * ny) return LBMICE_EINVAL;
    // stage the 9 float planes of each lattice in the free population buffer (it holds at
    // least 9 nx ny floats), then encode them into the current one; the h lattice's moment
    // is the phi^n plane, and with 16-bit storage U and rho are kept too
    float* stage = static_cast<float*>(h->pops[(s + 1) & 1]);
    for (int L = 0; L < h->nplanes / 9; ++L) {
      LB_TRY(cudaMemcpyAsync(stage, static_cast<const float*>(src) + (size_t)9 * L * nx * ny,
                             sizeof(float) * 9 * nx * ny, kind, h->stream));
      float* M = L == 0 ? h->phi[s % 3] : L == 1 ? h->Um[s & 1] : h->rhom[s & 1];
      int rc = with_storage(h, [&](auto tag) {
        using S = decltype(tag);
        encode_lattice_kernel<S><<<node_grid(h->C, blk), blk, 0, h->stream>>>(
            h->C, stage, L, h->pops[s & 1], M);
        return cuda_err(cudaGetLastError());
      });
      if (rc != LBMICE_OK) return rc;
    }
  } else {
    if (bytes < sizeof(float) * nx * ny) return LBMICE_EINVAL;
    LB_TRY(cudaMemcpy2DAsync(h->phi[(s + 2) % 3], h->C.pitch * sizeof(float), src,
                             nx * sizeof(float), nx * sizeof(float), ny, kind, h->stream));
  }
  if (!src_on_device) LB_TRY(cudaStreamSynchronize(h->stream));
  return LBMICE_OK;
}

extern "C" {

int lbmice_stats(lbmice_t* h, double out[LBMICE_NSTATS]) {
  if (!h || !out) return LBMICE_EINVAL;
  int rc = run_stats(h);
  if (rc != LBMICE_OK) return rc;
  for (int k = 0; k < kNStat; ++k) out[k] = h->stat_host[k];
  out[5] = (double)h->step;
  return LBMICE_OK;
}

int lbmice_tips(lbmice_t* h, double cx, double cy, double step, int32_t nrays,
                const double* angles_deg, double* radii) {
  if (!h || !angles_deg || !radii || nrays < 1 || nrays > LBMICE_MAX_RAYS ||
      !(step > 0.0) || !std::isfinite(step) || !std::isfinite(cx) || !std::isfinite(cy))
    return LBMICE_EINVAL;
  const double deg = 3.14159265358979323846 / 180.0;
  for (int i = 0; i < nrays; ++i) {
    if (!std::isfinite(angles_deg[i])) return LBMICE_EINVAL;
    h->tip_host[2 * i] = std::cos(angles_deg[i] * deg);
    h->tip_host[2 * i + 1] = std::sin(angles_deg[i] * deg);
  }
  double* cs = h->tip_dev;
  double* out = h->tip_dev + 2 * LBMICE_MAX_RAYS;
  LB_TRY(cudaMemcpyAsync(cs, h->tip_host, sizeof(double) * 2 * nrays, cudaMemcpyHostToDevice,
                         h->stream));
  const int per_block = 8;  // rays (warps) per block
  tips_kernel<<<(nrays + per_block - 1) / per_block, 32 * per_block, 0, h->stream>>>(
      h->phi[h->step % 3], h->C.nx, h->C.ny, h->C.pitch, cx, cy, step, nrays, cs, out);
  LB_TRY(cudaGetLastError());
  LB_TRY(cudaMemcpyAsync(h->tip_host + 2 * LBMICE_MAX_RAYS, out, sizeof(double) * nrays,
                         cudaMemcpyDeviceToHost, h->stream));
  LB_TRY(cudaStreamSynchronize(h->stream));
  for (int i = 0; i < nrays; ++i) radii[i] = h->tip_host[2 * LBMICE_MAX_RAYS + i];
  return LBMICE_OK;
}

int lbmice_sync(lbmice_t* h) {
  if (!h) return LBMICE_EINVAL;
  LB_TRY(cudaStreamSynchronize(h->stream));
  LB_TRY(cudaGetLastError());
  return LBMICE_OK;
}

int64_t lbmice_steps_done(const lbmice_t* h) { return h ? h->step : -1; }

int lbmice_destroy(lbmice_t* h) {
  if (!h) return LBMICE_OK;
  cudaError_t e = cudaStreamSynchronize(h->stream);
  release(h);
  return cuda_err(e);
}

const char* lbmice_last_error(void) { return g_last_cuda_error; }

const char* lbmice_strerror(int code) {
  switch (code) {
    case LBMICE_OK: return "ok";
    case LBMICE_EINVAL: return "invalid argument";
    case LBMICE_ECUDA: return "CUDA error";
    case LBMICE_ENOMEM: return "out of memory";
    case LBMICE_ENONFINITE: return "non-finite value in phi, U or rho";
    case LBMICE_EUNSTABLE: return "unstable parameters (relaxation time or inflow speed)";
    case LBMICE_ETIMEOUT: return "device-side wait timed out";
    case LBMICE_ENOTSUP: return "not supported by this build";
    default: return "unknown error";
  }
}

int lbmice_debug_flags(uint32_t* flags, int32_t clear) {
  if (!flags || (clear != 0 && clear != 1)) return LBMICE_EINVAL;
  *flags = 0;
#ifdef LBMICE_CHECKED
  LB_TRY(cudaDeviceSynchronize());  // every queued step, on any stream, has run
  unsigned w = 0;
  LB_TRY(cudaMemcpyFromSymbol(&w, lbmice::oob_word, sizeof(w)));
  *flags = w;
  if (clear) {
    const unsigned z = 0;
    LB_TRY(cudaMemcpyToSymbol(lbmice::oob_word, &z, sizeof(z)));
  }
  return LBMICE_OK;
#else
  return LBMICE_ENOTSUP;
#endif
}

int lbmice_debug_wait_selftest(void) {
  unsigned int w = 0;
  const unsigned int z = 0;
  LB_TRY(cudaDeviceSynchronize());
  LB_TRY(cudaMemcpyToSymbol(lbmice::wait_word, &z, sizeof(z)));
  lbmice::wait_selftest_kernel<<<1, 32>>>();
  LB_TRY(cudaGetLastError());
  LB_TRY(cudaDeviceSynchronize());
  LB_TRY(cudaMemcpyFromSymbol(&w, lbmice::wait_word, sizeof(w)));
  LB_TRY(cudaMemcpyToSymbol(lbmice::wait_word, &z, sizeof(z)));
  return w ? LBMICE_ETIMEOUT : LBMICE_OK;
}

int lbmice_debug_set_margin(int64_t margin) {
  if (margin < 0) return LBMICE_EINVAL;
#ifdef LBMICE_CHECKED
  LB_TRY(cudaDeviceSynchronize());
  const long long m = margin;
  LB_TRY(cudaMemcpyToSymbol(lbmice::oob_margin, &m, sizeof(m)));
  return LBMICE_OK;
#else
  return LBMICE_ENOTSUP;
#endif
}

}  // extern "C"

// ---------------------------------------------------------------------------------------
// FP64 diagnostics without allocation (declared in include/lbmice.h as lbmice_stats_noalloc).
//
// Some callers cannot allocate device memory at the moment they want these diagnostics:
// a host application whose device memory is reserved up front by its own pool allocator
// (so a cudaMalloc from this library would fail or fragment that budget), or a
// time-critical loop for which the implicit device synchronisation and unbounded latency of
// cudaMalloc/cudaFree are not acceptable. For them the per-block partial sums of the
// reduction live in the fixed array below, which every GPU that loads this library holds
// until the process exits.
// ---------------------------------------------------------------------------------------
namespace {

constexpr int kNoallocMaxBlocks = 2048;                  // partial rows in the fixed array
constexpr long long kNoallocNodesPerBlock = 8192;        // nodes summed by one block
constexpr int kNoallocMaxDevices = 64;
static_assert(kNoallocMaxBlocks * kNoallocNodesPerBlock == LBMICE_NOALLOC_MAX_NODES,
              "the fixed partial array must cover LBMICE_NOALLOC_MAX_NODES nodes");

// 2048 rows x 5 doubles = 80 KB. Every row a call reads is written by that same call before
// it is read, so nothing has to start at zero; the array keeps the last call's partials.
static __device__ __align__(256) double g_noalloc_partial[kNoallocMaxBlocks * kNStat];

std::atomic<double*> g_noalloc_ptr[kNoallocMaxDevices];

// Device address of the fixed array on the current device. Host code only holds a host-side
// stand-in for the symbol, so the address is asked for once per device, with that device
// current, and cached for the life of the process (valid while the device's primary context
// lives: a cudaDeviceReset makes it stale, as the header states).
int noalloc_scratch(double** out) {
  int dev = 0;
  LB_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNoallocMaxDevices) return LBMICE_EINVAL;
  double* p = g_noalloc_ptr[dev].load(std::memory_order_acquire);
  if (!p) {
    void* q = nullptr;
    LB_TRY(cudaGetSymbolAddress(&q, g_noalloc_partial));
    p = static_cast<double*>(q);
    g_noalloc_ptr[dev].store(p, std::memory_order_release);
  }
  *out = p;
  return LBMICE_OK;
}

}  // namespace

extern "C" int lbmice_stats_noalloc(const float* pops, const float* phi, const float* phi_prev,
                                    int32_t nx, int32_t ny, int32_t pitch, int32_t flow,
                                    double dx, double L_sat, double* out, void* stream) {
  if (!pops || !phi || !phi_prev || !out || nx < 1 || ny < 1 || pitch < nx ||
      (flow != 0 && flow != 1) || !(dx > 0) || !std::isfinite(L_sat))
    return LBMICE_EINVAL;
  const long long nodes = (long long)nx * ny;
  if (nodes > LBMICE_NOALLOC_MAX_NODES) return LBMICE_EINVAL;  // beyond the fixed array
  const int nblocks = (int)((nodes + kNoallocNodesPerBlock - 1) / kNoallocNodesPerBlock);
  double* partial = nullptr;
  int rc = noalloc_scratch(&partial);
  if (rc != LBMICE_OK) return rc;
  Consts C;
  std::memset(&C, 0, sizeof(C));
  C.nx = nx;
  C.ny = ny;
  C.pitch = pitch;
  C.pstride = (long long)pitch * ny;  // caller's layout: [plane][ny][pitch]
  C.rstride = pitch;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  stats_partial_kernel<F32P><<<nblocks, kStatThreads, 0, st>>>(
      C, flow, 0.5 * dx * dx, 0.5 * L_sat, pops, phi, phi_prev, nullptr, nullptr, partial);
  LB_TRY(cudaGetLastError());
  stats_final_kernel<<<1, 32, 0, st>>>(partial, nblocks, out);
  LB_TRY(cudaGetLastError());
  return LBMICE_OK;
}

// ---------------------------------------------------------------------------------------
// Batches: many member grids advanced by one launch per tile shape and step.
// ---------------------------------------------------------------------------------------
struct lbmice_batch {
  std::vector<lbmice_t*> members;
  std::vector<int> shape;             // tile shape id of each member
  cudaStream_t stream = nullptr;
  cudaStream_t capture = nullptr;     // private stream used only to record graphs
  int flow = 0, storage = 0;
  std::unique_ptr<BatchLaunch> block; // host scratch for one launch's parameter block
  cudaGraphExec_t graph = nullptr;
};

namespace {

// The batch has no step counter of its own: its members step together, and their common
// count (which re-initialising every member resets) decides the buffer phase.
int64_t batch_steps(const lbmice_batch_t* b) { return b->members[0]->step; }

// Work units of a member in a launch of this shape: tiles, or (strip, row) pairs of the march.
long long member_units(const lbmice_t* m, int shape) {
  if (shape == LBMICE_SHAPE_MARCH) return march_units(m->C, kMarchMaxSegRows);
  const int tx = shape_tx(shape), ty = shape_ty(shape);
  return (long long)((m->C.nx + tx - 1) / tx) * ((m->C.ny + ty - 1) / ty);
}

// Buffer roles of step phase ph (step mod 6), as the single-grid path rotates them.
// The region bases of a step's population buffers (StepPtrs::rin, rout): element offsets
// 4pQ (p = 0..3), 16Q, 18Q, 22Q, 26Q of an FP32 buffer, 9LQ (L = 0, 1, 2) of a 16-bit one.
void step_regions(StepPtrs& P, const Consts& C, bool dev16) {
  const long long Q = C.pstride;
  const long long f32_off[kRegions] = {0, 4 * Q, 8 * Q, 12 * Q, 16 * Q, 18 * Q, 22 * Q, 26 * Q};
  for (int r = 0; r < kRegions; ++r) {
    const long long bytes = dev16 ? (r < 3 ? 2 * 9 * r * Q : 0) : 4 * f32_off[r];
    const bool used = dev16 ? r < 3 : true;
    P.rin[r] = used ? static_cast<const char*>(P.pin) + bytes : nullptr;
    P.rout[r] = used ? static_cast<char*>(P.pout) + bytes : nullptr;
  }
}

StepPtrs step_ptrs(const lbmice_t* h, int ph) {
  StepPtrs P;
  P.pin = h->pops[ph & 1];
  P.pout = h->pops[(ph + 1) & 1];
  P.phi_n = h->phi[ph % 3];
  P.phi_nm1 = h->phi[(ph + 2) % 3];
  P.phi_np1 = h->phi[(ph + 1) % 3];
  P.U_n = h->Um[ph & 1];
  P.U_np1 = h->Um[(ph + 1) & 1];
  P.rho_n = h->rhom[ph & 1];
  P.rho_np1 = h->rhom[(ph + 1) & 1];
  P.tm = h->tmaps ? h->tmaps + kMapsPerPhase * ph : nullptr;
  step_regions(P, h->C, dev16(h));
  return P;
}

template <int TX, int TY>
int launch_block(const lbmice_batch_t* b, long long tiles, cudaStream_t st) {
  return with_storage(b->members[0], [&](auto tag) {
    using S = decltype(tag);
    if (b->flow)
      batch_step_kernel<TX, TY, true, S>
          <<<(unsigned)tiles, TX * TY, Tile<TX, TY>::template smem_bytes<true>(), st>>>(*b->block);
    else
      batch_step_kernel<TX, TY, false, S>
          <<<(unsigned)tiles, TX * TY, Tile<TX, TY>::template smem_bytes<false>(), st>>>(*b->block);
    return cuda_err(cudaGetLastError());
  });
}

int launch_march_block(const lbmice_batch_t* b, long long units, cudaStream_t st) {
  return with_storage(b->members[0], [&](auto tag) {
    using S = decltype(tag);
    // members with tensor maps (16-bit storage) prefetch, as their single-grid steps do
    constexpr int M = Storage<S>::DEV ? MARCH_PREFETCH : MARCH_PLAIN;
    if (b->flow)
      batch_march_kernel<true, S, M>
          <<<(unsigned)units, kMarchThreads, march_smem_bytes<true>(), st>>>(*b->block);
    else
      batch_march_kernel<false, S, M>
          <<<(unsigned)units, kMarchThreads, march_smem_bytes<false>(), st>>>(*b->block);
    return cuda_err(cudaGetLastError());
  });
}

// One step (phase ph) of the listed members: one launch per shape in use and per
// kBatchMaxMembers members of that shape.
int launch_members(lbmice_batch_t* b, const std::vector<int>& idx, int ph, cudaStream_t st) {
  for (int s = 0; s < kNumShapes; ++s) {
    size_t k = 0;
    while (true) {
      BatchLaunch& L = *b->block;
      L.n = 0;
      L.tile_start[0] = 0;
      for (; k < idx.size() && L.n < kBatchMaxMembers; ++k) {
        const int i = idx[k];
        if (b->shape[i] != s) continue;
        const lbmice_t* h = b->members[i];
        BatchDesc& d = L.d[L.n];
        d.C = h->C;
        d.C.seg_rows = kMarchMaxSegRows;
        d.P = step_ptrs(h, ph);
        d.tiles_x = s == LBMICE_SHAPE_MARCH ? march_strips(h->C.nx)
                                            : (h->C.nx + shape_tx(s) - 1) / shape_tx(s);
        d.pad_ = 0;
        L.tile_start[L.n + 1] = L.tile_start[L.n] + member_units(h, s);
        ++L.n;
      }
      if (L.n == 0) break;
      const long long units = L.tile_start[L.n];
      const int rc = s == LBMICE_SHAPE_MARCH  ? launch_march_block(b, units, st)
                     : s == LBMICE_SHAPE_32x8 ? launch_block<32, 8>(b, units, st)
                     : s == LBMICE_SHAPE_64x4 ? launch_block<64, 4>(b, units, st)
                                              : launch_block<16, 16>(b, units, st);
      if (rc != LBMICE_OK) return rc;
      if (k >= idx.size()) break;
    }
  }
  return LBMICE_OK;
}

void batch_release(lbmice_batch_t* b) {
  if (b->graph) cudaGraphExecDestroy(b->graph);
  for (lbmice_t* m : b->members) if (m) lbmice_destroy(m);
  if (b->capture) cudaStreamDestroy(b->capture);
  delete b;
}

std::vector<int> all_members(const lbmice_batch_t* b) {
  std::vector<int> v(b->members.size());
  for (size_t i = 0; i < v.size(); ++i) v[i] = (int)i;
  return v;
}

bool in_lockstep(const lbmice_batch_t* b) {
  for (const lbmice_t* m : b->members)
    if (m->step != batch_steps(b)) return false;
  return true;
}

void advance_members(lbmice_batch_t* b, int64_t n) {
  for (lbmice_t* m : b->members) m->step += n;
}

void drop_graph(lbmice_batch_t* b) {
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
}

}  // namespace

extern "C" {

int lbmice_batch_create(const lbmice_params* params, int32_t count, void* stream,
                        lbmice_batch_t** out) {
  if (!out) return LBMICE_EINVAL;
  *out = nullptr;
  if (!params || count < 1) return LBMICE_EINVAL;
  for (int i = 0; i < count; ++i) {
    if (params[i].flow != params[0].flow || params[i].storage != params[0].storage)
      return LBMICE_EINVAL;
    // the batched tile is the default one: E4 gradient, six-fold anisotropy
    if ((params[i].stencil != 0 && params[i].stencil != 4) ||
        (params[i].fold != 0 && params[i].fold != 6))
      return LBMICE_EINVAL;
    const int rc = validate(params[i]);
    if (rc != LBMICE_OK) return rc;
  }
  lbmice_batch_t* b = new (std::nothrow) lbmice_batch();
  if (!b) return LBMICE_ENOMEM;
  b->block.reset(new (std::nothrow) BatchLaunch());
  if (!b->block) {
    delete b;
    return LBMICE_ENOMEM;
  }
  b->stream = static_cast<cudaStream_t>(stream);
  b->flow = params[0].flow;
  b->storage = params[0].storage;
  b->members.assign(count, nullptr);
  b->shape.assign(count, LBMICE_SHAPE_MARCH);
  for (int i = 0; i < count; ++i) {
    const int rc = lbmice_create(&params[i], stream, &b->members[i]);
    if (rc != LBMICE_OK) {
      batch_release(b);
      return rc;
    }
  }
  const cudaError_t e = cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    batch_release(b);
    return cuda_err(e);
  }
  *out = b;
  return LBMICE_OK;
}

int32_t lbmice_batch_size(const lbmice_batch_t* b) { return b ? (int32_t)b->members.size() : 0; }

lbmice_t* lbmice_batch_member(lbmice_batch_t* b, int32_t i) {
  if (!b || i < 0 || i >= (int32_t)b->members.size()) return nullptr;
  return b->members[i];
}

int lbmice_batch_set_shape(lbmice_batch_t* b, int32_t i, int32_t shape) {
  if (!b || i < 0 || i >= (int32_t)b->members.size() || shape < 0 || shape >= kNumShapes)
    return LBMICE_EINVAL;
  b->shape[i] = shape;
  drop_graph(b);  // launches already queued keep the parameter blocks they were given
  return LBMICE_OK;
}

int lbmice_batch_step(lbmice_batch_t* b, int64_t nsteps) {
  if (!b || nsteps < 0) return LBMICE_EINVAL;
  if (!in_lockstep(b)) return LBMICE_EINVAL;
  const std::vector<int> all = all_members(b);
  int64_t left = nsteps;
  while (left > 0) {
    if (batch_steps(b) % 6 == 0 && left >= kGraphSteps) {
      if (!b->graph) {
        cudaGraph_t g = nullptr;
        LB_TRY(cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal));
        int rc = LBMICE_OK;
        for (int s = 0; s < kGraphSteps && rc == LBMICE_OK; ++s)
          rc = launch_members(b, all, s % 6, b->capture);
        cudaError_t e = cudaStreamEndCapture(b->capture, &g);
        if (rc != LBMICE_OK) { if (g) cudaGraphDestroy(g); return rc; }
        if (e != cudaSuccess) return cuda_err(e);
        e = cudaGraphInstantiate(&b->graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) { b->graph = nullptr; return cuda_err(e); }
      }
      LB_TRY(cudaGraphLaunch(b->graph, b->stream));
      advance_members(b, kGraphSteps);
      left -= kGraphSteps;
    } else {
      const int rc = launch_members(b, all, (int)(batch_steps(b) % 6), b->stream);
      if (rc != LBMICE_OK) return rc;
      advance_members(b, 1);
      left -= 1;
    }
  }
  return LBMICE_OK;
}

int lbmice_batch_autotune(lbmice_batch_t* b, int32_t steps_per_trial, int32_t* shapes,
                          int64_t* steps_taken) {
  if (!b || steps_per_trial < 1) return LBMICE_EINVAL;
  if (!in_lockstep(b)) return LBMICE_EINVAL;
  const int n = (int)b->members.size();
  drop_graph(b);
  // size classes
  std::vector<std::pair<int, int>> classes;
  for (const lbmice_t* m : b->members) {
    const std::pair<int, int> key(m->C.nx, m->C.ny);
    if (std::find(classes.begin(), classes.end(), key) == classes.end()) classes.push_back(key);
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  LB_TRY(cudaEventCreate(&e0));
  LB_TRY(cudaEventCreate(&e1));
  int64_t taken = 0;
  int rc = LBMICE_OK;
  for (const auto& cls : classes) {
    std::vector<int> in, rest;
    for (int i = 0; i < n; ++i)
      (b->members[i]->C.nx == cls.first && b->members[i]->C.ny == cls.second ? in : rest)
          .push_back(i);
    float best = 0.0f;
    int best_shape = 0;
    for (int s = 0; s < kNumShapes && rc == LBMICE_OK; ++s) {
      for (int i : in) b->shape[i] = s;
      // one untimed step, then the timed steps of this class; the other members take the
      // same number of steps untimed, so the batch stays in lockstep
      const int64_t base = batch_steps(b);
      for (int k = 0; k <= steps_per_trial && rc == LBMICE_OK; ++k) {
        if (k == 1) rc = cuda_err(cudaEventRecord(e0, b->stream));
        if (rc == LBMICE_OK) rc = launch_members(b, in, (int)((base + k) % 6), b->stream);
      }
      if (rc == LBMICE_OK) rc = cuda_err(cudaEventRecord(e1, b->stream));
      for (int k = 0; k <= steps_per_trial && rc == LBMICE_OK && !rest.empty(); ++k)
        rc = launch_members(b, rest, (int)((base + k) % 6), b->stream);
      if (rc == LBMICE_OK) rc = cuda_err(cudaStreamSynchronize(b->stream));
      float ms = 0.0f;
      if (rc == LBMICE_OK) rc = cuda_err(cudaEventElapsedTime(&ms, e0, e1));
      if (rc == LBMICE_OK) {
        advance_members(b, steps_per_trial + 1);
        taken += steps_per_trial + 1;
        if (s == 0 || ms < best) {
          best = ms;
          best_shape = s;
        }
      }
    }
    for (int i : in) b->shape[i] = best_shape;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != LBMICE_OK) return rc;
  if (shapes)
    for (int i = 0; i < n; ++i) shapes[i] = b->shape[i];
  if (steps_taken) *steps_taken = taken;
  return LBMICE_OK;
}

int lbmice_batch_destroy(lbmice_batch_t* b) {
  if (!b) return LBMICE_OK;
  cudaError_t e = cudaStreamSynchronize(b->stream);
  batch_release(b);
  return cuda_err(e);
}

}  // extern "C"

// ---------------------------------------------------------------------------------------
// Tape: a checkpointed forward record of one grid and the discrete adjoint of its steps
// (periodic faces, FP32 storage). Checkpoints are state blobs every `every` steps; the
// reverse sweep restores each segment's checkpoint, recomputes the segment's states with the
// step kernel and runs the adjoint kernels backwards through them.
// ---------------------------------------------------------------------------------------
struct lbmice_tape {
  lbmice_t* h = nullptr;           // the recorded grid (borrowed)
  int every = 100;                 // checkpoint interval
  int64_t steps = 0;               // steps recorded
  std::vector<void*> ckpt;         // states at steps 0, every, 2 every, ...
  // reverse-sweep work space, allocated by the first backward
  std::vector<float*> seg_pops;    // every + 1 population buffers: states of one segment
  std::vector<float*> seg_phi;     // every + 2 phi planes: phi^{s0-1}, phi^{s0}, ...
  float* pb[2] = {nullptr, nullptr};
  float* Phib[2] = {nullptr, nullptr};
  float* Psib[2] = {nullptr, nullptr};
  std::vector<float*> plane;       // scratch planes, see enum below
  double* partial = nullptr;       // [blocks][kAdjParams]
  int nblocks = 0;
  // the pull's own-population term inside the collision adjoint (grids whose reverse working
  // set, about 4 x 116 B per node, exceeds the L2), else in a separate read-modify-write pass
  bool fused = false;
  // a full segment's recompute and reverse steps as a CUDA graph, one per starting parity of
  // the adjoint ping-pong (every argument is the same for every full segment)
  cudaGraphExec_t seg_graph[2] = {nullptr, nullptr};
};

namespace {

enum : int {
  TP_PHIB_LOC = 0, TP_GBX, TP_GBY, TP_BN, TP_SEED_PHI, TP_SEED_U, TP_PHI0B, TP_U0B, TP_RHO0B,
  TP_UX0B, TP_UY0B, TP_NPLANES
};

bool tape_supported(const lbmice_t* h) {
  if (h->p.storage != LBMICE_STORAGE_F32) return false;
  for (int f = 0; f < 4; ++f)
    if (h->p.bc[f] != LBMICE_BC_PERIODIC) return false;
  return true;
}

// State blob of the current step, kept when the step is a multiple of the interval.
int tape_checkpoint(lbmice_tape_t* t) {
  const size_t c = (size_t)(t->steps / t->every);
  if (c < t->ckpt.size()) return LBMICE_OK;
  void* blob = nullptr;
  LB_TRY(cudaMalloc(&blob, lbmice_state_bytes(t->h)));
  t->ckpt.push_back(blob);
  return copy_state(t->h, blob, true, cudaMemcpyDeviceToDevice);
}

int tape_alloc_work(lbmice_tape_t* t) {
  if (t->partial) return LBMICE_OK;
  const lbmice_t* h = t->h;
  auto grab = [](size_t bytes, float** p) { return cudaMalloc(reinterpret_cast<void**>(p), bytes); };
  t->seg_pops.assign(t->every + 1, nullptr);
  t->seg_phi.assign(t->every + 2, nullptr);
  t->plane.assign(TP_NPLANES, nullptr);
  cudaError_t e = cudaSuccess;
  for (float*& b : t->seg_pops) if (e == cudaSuccess) e = grab(pop_bytes(h), &b);
  for (float*& b : t->seg_phi) if (e == cudaSuccess) e = grab(field_bytes(h), &b);
  for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
    e = grab(pop_bytes(h), &t->pb[k]);
    if (e == cudaSuccess) e = grab(field_bytes(h), &t->Phib[k]);
    if (e == cudaSuccess) e = grab(field_bytes(h), &t->Psib[k]);
  }
  for (float*& b : t->plane) if (e == cudaSuccess) e = grab(field_bytes(h), &b);
  t->nblocks = ((h->C.nx + 31) / 32) * ((h->C.ny + 7) / 8);
  if (e == cudaSuccess)
    e = cudaMalloc(reinterpret_cast<void**>(&t->partial),
                   sizeof(double) * kAdjParams * t->nblocks);
  for (float* b : t->plane)  // planes are read over their full pitch by the copies out
    if (e == cudaSuccess && b) e = cudaMemsetAsync(b, 0, field_bytes(h), h->stream);
  return cuda_err(e);
}

void tape_free(lbmice_tape_t* t) {
  for (cudaGraphExec_t g : t->seg_graph) if (g) cudaGraphExecDestroy(g);
  for (void* b : t->ckpt) cudaFree(b);
  for (float* b : t->seg_pops) if (b) cudaFree(b);
  for (float* b : t->seg_phi) if (b) cudaFree(b);
  for (int k = 0; k < 2; ++k) {
    if (t->pb[k]) cudaFree(t->pb[k]);
    if (t->Phib[k]) cudaFree(t->Phib[k]);
    if (t->Psib[k]) cudaFree(t->Psib[k]);
  }
  for (float* b : t->plane) if (b) cudaFree(b);
  if (t->partial) cudaFree(t->partial);
  delete t;
}

// Checkpoint c into the first state of the segment buffers (blob: populations, phi^n,
// phi^{n-1}, as copy_state writes it for FP32 storage).
int tape_restore(lbmice_tape_t* t, size_t c) {
  const lbmice_t* h = t->h;
  const char* b = static_cast<const char*>(t->ckpt[c]);
  LB_TRY(cudaMemcpyAsync(t->seg_pops[0], b, pop_bytes(h), cudaMemcpyDeviceToDevice, h->stream));
  b += pop_bytes(h);
  LB_TRY(cudaMemcpyAsync(t->seg_phi[1], b, field_bytes(h), cudaMemcpyDeviceToDevice,
                         h->stream));
  b += field_bytes(h);
  LB_TRY(cudaMemcpyAsync(t->seg_phi[0], b, field_bytes(h), cudaMemcpyDeviceToDevice,
                         h->stream));
  return LBMICE_OK;
}

StepPtrs tape_step_ptrs(const lbmice_tape_t* t, int j) {
  StepPtrs P{};
  P.pin = t->seg_pops[j];
  P.pout = t->seg_pops[j + 1];
  P.phi_n = t->seg_phi[j + 1];
  P.phi_nm1 = t->seg_phi[j];
  P.phi_np1 = t->seg_phi[j + 2];
  step_regions(P, t->h->C, dev16(t->h));
  return P;
}

dim3 adj_grid(const lbmice_t* h) { return dim3((h->C.nx + 31) / 32, (h->C.ny + 7) / 8); }

// Reverse step through segment state j: adjoint buffers cur -> 1 - cur.
int tape_reverse_step(lbmice_tape_t* t, int j, int cur, cudaStream_t st) {
  const lbmice_t* h = t->h;
  AdjPtrs A;
  A.pops = t->seg_pops[j];
  A.phi_n = t->seg_phi[j + 1];
  A.phi_nm1 = t->seg_phi[j];
  A.pb_in = t->pb[cur];
  A.Phib_in = t->Phib[cur];
  A.Psib_in = t->Psib[cur];
  A.pb_out = t->pb[1 - cur];
  A.Phib_out = t->Phib[1 - cur];
  A.Psib_out = t->Psib[1 - cur];
  A.phib_loc = t->plane[TP_PHIB_LOC];
  A.gbx = t->plane[TP_GBX];
  A.gby = t->plane[TP_GBY];
  A.Bn = t->plane[TP_BN];
  A.partial = t->partial;
  const dim3 g = adj_grid(h);
  if (t->fused) {
    adj_b_kernel<<<g, 256, 0, st>>>(h->C, A);
    if (h->p.flow)
      adj_collide_kernel<true, true><<<g, 256, 0, st>>>(h->C, A);
    else
      adj_collide_kernel<false, true><<<g, 256, 0, st>>>(h->C, A);
    adj_stencil_kernel<<<g, 256, 0, st>>>(h->C, A);
  } else {
    if (h->p.flow)
      adj_collide_kernel<true, false><<<g, 256, 0, st>>>(h->C, A);
    else
      adj_collide_kernel<false, false><<<g, 256, 0, st>>>(h->C, A);
    adj_pull_kernel<<<g, 256, 0, st>>>(h->C, A);
  }
  return cuda_err(cudaGetLastError());
}

// Recompute the states of a segment of len steps from its restored first state, then run
// the reverse steps through them, starting from adjoint buffer cur.
int tape_segment(lbmice_tape_t* t, int len, int cur, cudaStream_t st) {
  int rc = LBMICE_OK;
  for (int j = 0; j + 1 < len && rc == LBMICE_OK; ++j)
    rc = launch_step_ptrs(t->h, tape_step_ptrs(t, j), st);
  for (int j = len - 1; j >= 0 && rc == LBMICE_OK; --j) {
    rc = tape_reverse_step(t, j, cur, st);
    cur = 1 - cur;
  }
  return rc;
}

// [ny][nx] float array (host or device) <-> [ny][pitch] plane.
int plane_in(const lbmice_t* h, float* plane, const float* src) {
  const size_t w = sizeof(float) * h->C.nx;
  LB_TRY(cudaMemcpy2DAsync(plane, sizeof(float) * h->C.pitch, src, w, w, h->C.ny,
                           cudaMemcpyDefault, h->stream));
  return LBMICE_OK;
}
int plane_out(const lbmice_t* h, float* dst, const float* plane) {
  const size_t w = sizeof(float) * h->C.nx;
  LB_TRY(cudaMemcpy2DAsync(dst, w, plane, sizeof(float) * h->C.pitch, w, h->C.ny,
                           cudaMemcpyDefault, h->stream));
  return LBMICE_OK;
}

}  // namespace

extern "C" {

int lbmice_tape_create(lbmice_t* h, int32_t every, lbmice_tape_t** out) {
  if (!out) return LBMICE_EINVAL;
  *out = nullptr;
  if (!h || every < 1 || !tape_supported(h) || h->step != 0) return LBMICE_EINVAL;
  if (h->C.stencil != 4 || h->C.fold != 6) return LBMICE_EINVAL;  // the adjoint's E4, six-fold
  lbmice_tape_t* t = new (std::nothrow) lbmice_tape();
  if (!t) return LBMICE_ENOMEM;
  t->h = h;
  t->every = every;
  {
    // the fused reverse pull for grids whose reverse working set exceeds the L2;
    // LBMICE_ADJ_FUSED=0 or 1 in the environment forces one form (both give the same bits)
    int l2 = 0;
    if (cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, h->device) != cudaSuccess) l2 = 0;
    t->fused = 4.0 * 116.0 * (double)h->C.nx * (double)h->C.ny > (double)l2;
    if (const char* e = std::getenv("LBMICE_ADJ_FUSED")) {
      if (e[0] == '0' && e[1] == 0) t->fused = false;
      if (e[0] == '1' && e[1] == 0) t->fused = true;
    }
  }
  const int rc = tape_checkpoint(t);
  if (rc != LBMICE_OK) {
    tape_free(t);
    return rc;
  }
  *out = t;
  return LBMICE_OK;
}

int64_t lbmice_tape_steps(const lbmice_tape_t* t) { return t ? t->steps : -1; }

int lbmice_tape_record(lbmice_tape_t* t, int64_t nsteps) {
  if (!t || nsteps < 0) return LBMICE_EINVAL;
  if (t->h->step != t->steps) return LBMICE_EINVAL;  // stepped outside the tape
  int64_t left = nsteps;
  while (left > 0) {
    const int64_t chunk = std::min<int64_t>(left, t->every - t->steps % t->every);
    const int rc = lbmice_step(t->h, chunk);
    t->steps = t->h->step;
    if (rc != LBMICE_OK) return rc;
    left -= chunk;
    if (t->steps % t->every == 0) {
      const int rc2 = tape_checkpoint(t);
      if (rc2 != LBMICE_OK) return rc2;
    }
  }
  return LBMICE_OK;
}

int lbmice_tape_backward(lbmice_tape_t* t, const float* phi_bar, const float* U_bar,
                         double grads[3], float* phi0_bar, float* U0_bar, float* rho0_bar,
                         float* ux0_bar, float* uy0_bar) {
  if (!t) return LBMICE_EINVAL;
  lbmice_t* h = t->h;
  if (h->step != t->steps) return LBMICE_EINVAL;
  int rc = tape_alloc_work(t);
  if (rc != LBMICE_OK) return rc;
  const dim3 g = adj_grid(h);
  // seed: dL/dphi_T into the phi-plane adjoint, dL/dU_T into the g adjoints
  if (phi_bar && (rc = plane_in(h, t->plane[TP_SEED_PHI], phi_bar)) != LBMICE_OK) return rc;
  if (U_bar && (rc = plane_in(h, t->plane[TP_SEED_U], U_bar)) != LBMICE_OK) return rc;
  const float* sp = phi_bar ? t->plane[TP_SEED_PHI] : nullptr;
  const float* su = U_bar ? t->plane[TP_SEED_U] : nullptr;
  if (h->p.flow)
    adj_seed_kernel<true><<<g, 256, 0, h->stream>>>(h->C, sp, su, t->pb[0], t->Phib[0],
                                                    t->Psib[0]);
  else
    adj_seed_kernel<false><<<g, 256, 0, h->stream>>>(h->C, sp, su, t->pb[0], t->Phib[0],
                                                     t->Psib[0]);
  LB_TRY(cudaGetLastError());
  LB_TRY(cudaMemsetAsync(t->partial, 0, sizeof(double) * kAdjParams * t->nblocks, h->stream));
  int cur = 0;
  // segments from the last: restore, recompute its states, reverse through them
  const int64_t nseg = (t->steps + t->every - 1) / t->every;
  for (int64_t c = nseg - 1; c >= 0; --c) {
    const int64_t s0 = c * t->every;
    const int len = (int)std::min<int64_t>(t->every, t->steps - s0);
    if ((rc = tape_restore(t, (size_t)c)) != LBMICE_OK) return rc;
    if (len == t->every) {  // a full segment: replay its graph
      if (!t->seg_graph[cur]) {
        cudaGraph_t gr = nullptr;
        LB_TRY(cudaStreamBeginCapture(h->capture, cudaStreamCaptureModeThreadLocal));
        rc = tape_segment(t, len, cur, h->capture);
        const cudaError_t e = cudaStreamEndCapture(h->capture, &gr);
        if (rc != LBMICE_OK) { if (gr) cudaGraphDestroy(gr); return rc; }
        if (e != cudaSuccess) return cuda_err(e);
        const cudaError_t ei = cudaGraphInstantiate(&t->seg_graph[cur], gr, 0);
        cudaGraphDestroy(gr);
        if (ei != cudaSuccess) { t->seg_graph[cur] = nullptr; return cuda_err(ei); }
      }
      LB_TRY(cudaGraphLaunch(t->seg_graph[cur], h->stream));
    } else if ((rc = tape_segment(t, len, cur, h->stream)) != LBMICE_OK) {
      return rc;
    }
    if (len & 1) cur = 1 - cur;
  }
  if (nseg == 0 && (rc = tape_restore(t, 0)) != LBMICE_OK) return rc;
  // initial state: adjoints of the moments it was built from
  InitAdjPtrs I;
  I.pops = t->seg_pops[0];
  I.phi0 = t->seg_phi[1];
  I.pb = t->pb[cur];
  I.Phib = t->Phib[cur];
  I.Psib = t->Psib[cur];
  I.phib_loc = t->plane[TP_PHIB_LOC];
  I.gbx = t->plane[TP_GBX];
  I.gby = t->plane[TP_GBY];
  I.Ub = t->plane[TP_U0B];
  I.rhob = t->plane[TP_RHO0B];
  I.uxb = t->plane[TP_UX0B];
  I.uyb = t->plane[TP_UY0B];
  I.partial = t->partial;
  if (h->p.flow)
    adj_init_kernel<true><<<g, 256, 0, h->stream>>>(h->C, I);
  else
    adj_init_kernel<false><<<g, 256, 0, h->stream>>>(h->C, I);
  adj_gather_kernel<<<g, 256, 0, h->stream>>>(h->C, t->plane[TP_PHIB_LOC], t->plane[TP_GBX],
                                              t->plane[TP_GBY], t->plane[TP_PHI0B]);
  LB_TRY(cudaGetLastError());
  const float* outs[5] = {t->plane[TP_PHI0B], t->plane[TP_U0B], t->plane[TP_RHO0B],
                          t->plane[TP_UX0B], t->plane[TP_UY0B]};
  float* dsts[5] = {phi0_bar, U0_bar, rho0_bar, ux0_bar, uy0_bar};
  for (int k = 0; k < 5; ++k)
    if (dsts[k] && (rc = plane_out(h, dsts[k], outs[k])) != LBMICE_OK) return rc;
  std::vector<double> part((size_t)kAdjParams * t->nblocks);
  LB_TRY(cudaMemcpyAsync(part.data(), t->partial, sizeof(double) * part.size(),
                         cudaMemcpyDeviceToHost, h->stream));
  LB_TRY(cudaStreamSynchronize(h->stream));
  double sum[kAdjParams] = {0.0, 0.0, 0.0, 0.0};
  for (int b = 0; b < t->nblocks; ++b)
    for (int k = 0; k < kAdjParams; ++k) sum[k] += part[(size_t)b * kAdjParams + k];
  if (grads) {
    const lbmice_params& p = h->p;
    // eps enters as eps and as kappa_N 6 eps; D as D_lat3 = 3 D dt/dx^2 and, when lambda is
    // not given, through the beta = 0 lambda = tau0 D / (a2 W0^2) (Sec. 2.1)
    grads[0] = sum[ADJ_EPS] + 6.0 * p.kappa_N * sum[ADJ_KN6EPS];
    grads[1] = sum[ADJ_DLAT3] * 3.0 * p.dt / (p.dx * p.dx);
    if (!(p.lambda > 0)) grads[1] += sum[ADJ_LAMBDA] * p.tau0 / (kA2 * p.W0 * p.W0);
    grads[2] = sum[ADJ_LAMBDA];
  }
  return LBMICE_OK;
}

int lbmice_tape_destroy(lbmice_tape_t* t) {
  if (!t) return LBMICE_OK;
  const cudaError_t e = cudaStreamSynchronize(t->h->stream);
  tape_free(t);
  return cuda_err(e);
}

}  // extern "C"
