// Device code of the coupled lattice-Boltzmann ice-crystal step (arXiv 2101.07163, Sec. 2.2)
// for sm_103a: the fused collide-stream kernel over the three D2Q9 lattices, the
// equilibrium initialisation, the moment export and the FP64 reductions.
//
// State layout in HBM (one allocation per buffer, row pitch padded to 32 elements):
//   populations: 27 planes of pstride elements, two buffers (the pull reads one and writes
//                the other), node-interleaved (load_hg_f32 and friends below). FP32 keeps the
//                phase-field and vapour populations of a node paired, (h_a, g_a), in four
//                float4 and a float2 (planes 0..17), and the flow populations as two float4
//                and a float (planes 18..26); 16-bit storage keeps the 8 deviations of a node
//                and lattice as one 16-byte vector in each of the regions [h | g | f];
//   phi:         three rotating [ny][pitch] float planes holding phi^{n-1}, phi^n, phi^{n+1}
//                (phi^n feeds the E4 gradient with a two-node halo, phi^{n-1} the d(phi)/dt
//                of the vapour source, phi^{n+1} = sum h^{n+1} is written by the step).
// Node (x, y) is node index y * rstride + x; the exported layout [q][ny][nx] puts population q
// of that node at q * nx ny + y * nx + x.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace lbmice {

// ---- checked build ----------------------------------------------------------------------
// Compiled with -DLBMICE_CHECKED (liblbmice_checked.so), the step kernels test every global
// and shared-memory index against the extent of its buffer before the access, in place of a
// memory checker: a violation sets a bit of the device word oob_word and the access is
// skipped (a load gives 0), so nothing traps. oob_margin shrinks every extent the tests use
// by that many elements, so that a test can see the checks fire on accesses that are still
// inside their buffers. In the normal build every test is the constant true and compiles
// away.
enum : unsigned { OOB_POPS = 1u, OOB_PLANE = 2u, OOB_SHARED = 4u };
#ifdef LBMICE_CHECKED
__device__ unsigned int oob_word;
__device__ long long oob_margin;
__device__ __forceinline__ bool in_range(long long i, long long n, unsigned bit) {
  if (i >= 0 && i < n - oob_margin) return true;
  atomicOr(&oob_word, bit);
  return false;
}
#else
__device__ __forceinline__ constexpr bool in_range(long long, long long, unsigned) {
  return true;
}
#endif

// ---- D2Q9 (directions are compile-time after unrolling) ---------------------------------
__host__ __device__ constexpr int cx_of(int a) {
  return (a == 1 || a == 5 || a == 8) ? 1 : ((a == 3 || a == 6 || a == 7) ? -1 : 0);
}
__host__ __device__ constexpr int cy_of(int a) {
  return (a == 2 || a == 5 || a == 6) ? 1 : ((a == 4 || a == 7 || a == 8) ? -1 : 0);
}
__host__ __device__ constexpr float w_of(int a) {
  return a == 0 ? 4.0f / 9.0f : (a < 5 ? 1.0f / 9.0f : 1.0f / 36.0f);
}
__host__ __device__ constexpr double wd_of(int a) {
  return a == 0 ? 4.0 / 9.0 : (a < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
}
// direction index after reflecting c_x (mirror across a vertical wall) or c_y
__host__ __device__ constexpr int mirx_of(int a) {
  return a == 1 ? 3 : a == 3 ? 1 : a == 5 ? 6 : a == 6 ? 5 : a == 7 ? 8 : a == 8 ? 7 : a;
}
__host__ __device__ constexpr int miry_of(int a) {
  return a == 2 ? 4 : a == 4 ? 2 : a == 5 ? 8 : a == 8 ? 5 : a == 6 ? 7 : a == 7 ? 6 : a;
}

// c_a . v built from additions and exact negations only, so the mirror image of a state
// produces bit-identical projections.
template <class T>
__device__ __forceinline__ T cdot(int a, T vx, T vy) {
  const int cx = cx_of(a), cy = cy_of(a);
  if (cx == 0) return cy > 0 ? vy : (cy < 0 ? -vy : T(0));
  const T r = cx > 0 ? vx : -vx;
  if (cy == 0) return r;
  return cy > 0 ? r + vy : r - vy;
}

// Sums over the nine directions grouped by opposite pairs; invariant under every
// reflection of the square, which keeps mirror-symmetric states bit-exactly symmetric.
template <class T>
__device__ __forceinline__ T sum9(const T* v) {
  return v[0] + (((v[1] + v[3]) + (v[2] + v[4])) + ((v[5] + v[7]) + (v[6] + v[8])));
}
template <class T>
__device__ __forceinline__ T sumcx9(const T* v) {
  return (v[1] - v[3]) + ((v[5] - v[7]) + (v[8] - v[6]));
}
template <class T>
__device__ __forceinline__ T sumcy9(const T* v) {
  return (v[2] - v[4]) + ((v[5] - v[7]) + (v[6] - v[8]));
}

// ---- storage of the populations ------------------------------------------------------
// F32: the 9 populations of each lattice as float. F16 / BF16: the zeroth moment M of each
// lattice as float (phi for h, U for g, rho for f, each in its own [ny][pitch] array) and the
// 8 moving populations as 16-bit deviations d_a = p_a - w_a M (node-interleaved, below); the
// rest population is rebuilt
// as p_0 = M - sum_{a>0} p_a (summed in the pairing of sum9), so the populations sum back to
// the stored M whatever the rounding of the deviations -- no systematic drift of mass or of
// the vapour invariant. All arithmetic is FP32.
struct F32 {};
struct F16 {};
struct BF16 {};
struct F32P {};  // FP32 populations in the exported plane layout (caller-owned diagnostics)
template <class S> struct Storage;
template <> struct Storage<F32> {
  using T = float;
  static constexpr bool DEV = false;
  static constexpr bool PLANES = false;
};
template <> struct Storage<F32P> {
  using T = float;
  static constexpr bool DEV = false;
  static constexpr bool PLANES = true;
};
// 16-bit forms: the 8 deviations of one node and lattice are 16 contiguous bytes, moved by
// one 128-bit load or store and converted in pairs (round to nearest).
template <> struct Storage<F16> {
  using T = __half;
  static constexpr bool DEV = true;
  static constexpr bool PLANES = false;
  __device__ static __forceinline__ void unpack8(const uint4& v, float* d) {
    const __half2* h = reinterpret_cast<const __half2*>(&v);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float2 f = __half22float2(h[k]);
      d[2 * k] = f.x;
      d[2 * k + 1] = f.y;
    }
  }
  __device__ static __forceinline__ uint4 pack8(const float* d) {
    uint4 v;
    __half2* h = reinterpret_cast<__half2*>(&v);
#pragma unroll
    for (int k = 0; k < 4; ++k) h[k] = __floats2half2_rn(d[2 * k], d[2 * k + 1]);
    return v;
  }
};
template <> struct Storage<BF16> {
  using T = __nv_bfloat16;
  static constexpr bool DEV = true;
  static constexpr bool PLANES = false;
  __device__ static __forceinline__ void unpack8(const uint4& v, float* d) {
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&v);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float2 f = __bfloat1622float2(h[k]);
      d[2 * k] = f.x;
      d[2 * k + 1] = f.y;
    }
  }
  __device__ static __forceinline__ uint4 pack8(const float* d) {
    uint4 v;
    __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(&v);
#pragma unroll
    for (int k = 0; k < 4; ++k) h[k] = __floats2bfloat162_rn(d[2 * k], d[2 * k + 1]);
    return v;
  }
};

// Addressing of the populations, with Q = pstride and node = y * rstride + x.
//   F32: the phase-field and vapour populations in pairs (h_a, g_a): directions 1, 2 of the
//     node as one float4 (h_1, g_1, h_2, g_2) at element 4 node, directions 3, 4 at
//     4 Q + 4 node, 5, 6 at 8 Q + 4 node, 7, 8 at 12 Q + 4 node, the rest pair (h_0, g_0) as a
//     float2 at 16 Q + 2 node; the flow populations from element 18 Q: directions 1..4 as one
//     float4 at 4 node, 5..8 at 4 Q + 4 node, the rest population at 8 Q + node;
//   F16 / BF16: lattice L (0 h, 1 g, 2 f) owns elements 9 L Q .. 9 (L + 1) Q; the 8
//     deviations a = 1..8 of the node at 8 node + (a - 1), the rest population not stored;
//   F32P (diagnostics of caller-owned exports only): population a of lattice L at
//     (9 L + a) Q + node.
// Every vector is aligned to its size because the pitch is a multiple of 32 elements; a
// warp's 32 nodes move as contiguous 256- or 512-byte runs per vector.

// Element offset of population a of lattice L at a node within an FP32 buffer.
__device__ __forceinline__ long long f32_pop_index(long long Q, long long node, int L, int a) {
  if (L == 2)
    return 18 * Q + (a == 0 ? 8 * Q + node : (a < 5 ? 4 * node + (a - 1) : 4 * Q + 4 * node + (a - 5)));
  if (a == 0) return 16 * Q + 2 * node + L;
  return 4 * Q * ((a - 1) >> 1) + 4 * node + 2 * ((a - 1) & 1) + L;
}

// The phase-field and vapour populations of an FP32 node as pairs hg[a] = (h_a, g_a).
__device__ __forceinline__ void load_hg_f32(const float* __restrict__ pops, long long Q,
                                            long long node, float2* hg) {
  if (!in_range(node, Q, OOB_POPS)) {
#pragma unroll
    for (int a = 0; a < 9; ++a) hg[a] = make_float2(0.0f, 0.0f);
    return;
  }
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(pops + 4 * p * Q + 4 * node));
    hg[2 * p + 1] = make_float2(v.x, v.y);
    hg[2 * p + 2] = make_float2(v.z, v.w);
  }
  hg[0] = __ldg(reinterpret_cast<const float2*>(pops + 16 * Q + 2 * node));
}
__device__ __forceinline__ void store_hg_f32(float* __restrict__ pops, long long Q,
                                             long long node, const float2* hg) {
  if (!in_range(node, Q, OOB_POPS)) return;
#pragma unroll
  for (int p = 0; p < 4; ++p)
    *reinterpret_cast<float4*>(pops + 4 * p * Q + 4 * node) =
        make_float4(hg[2 * p + 1].x, hg[2 * p + 1].y, hg[2 * p + 2].x, hg[2 * p + 2].y);
  *reinterpret_cast<float2*>(pops + 16 * Q + 2 * node) = hg[0];
}

// The 9 FP32 flow populations at a node; lat points at the flow region (element 18 Q).
__device__ __forceinline__ void load_lattice_f32(const float* __restrict__ lat, long long pstride,
                                                 long long node, float* out) {
  if (!in_range(node, pstride, OOB_POPS)) {
#pragma unroll
    for (int a = 0; a < 9; ++a) out[a] = 0.0f;
    return;
  }
  const float4 p = __ldg(reinterpret_cast<const float4*>(lat + 4 * node));
  const float4 q = __ldg(reinterpret_cast<const float4*>(lat + 4 * pstride + 4 * node));
  out[0] = __ldg(lat + 8 * pstride + node);
  out[1] = p.x;
  out[2] = p.y;
  out[3] = p.z;
  out[4] = p.w;
  out[5] = q.x;
  out[6] = q.y;
  out[7] = q.z;
  out[8] = q.w;
}
__device__ __forceinline__ void store_lattice_f32(float* __restrict__ lat, long long pstride,
                                                  long long node, const float* v) {
  if (!in_range(node, pstride, OOB_POPS)) return;
  *reinterpret_cast<float4*>(lat + 4 * node) = make_float4(v[1], v[2], v[3], v[4]);
  *reinterpret_cast<float4*>(lat + 4 * pstride + 4 * node) = make_float4(v[5], v[6], v[7], v[8]);
  lat[8 * pstride + node] = v[0];
}

// The 9 populations of one node and lattice from its 16-bit deviation vector v and its
// zeroth moment M: p_a = w_a M + d_a for a > 0, and the rest population from the sum.
template <class S>
__device__ __forceinline__ void decode9(uint4 v, float M, float* out) {
  float d[8];
  Storage<S>::unpack8(v, d);
#pragma unroll
  for (int a = 1; a < 9; ++a) out[a] = fmaf(a < 5 ? 1.0f / 9.0f : 1.0f / 36.0f, M, d[a - 1]);
  out[0] =
      M - (((out[1] + out[3]) + (out[2] + out[4])) + ((out[5] + out[7]) + (out[6] + out[8])));
}

// Checked raw accesses: the 16-byte deviation vector of node `node` of a lattice region (n
// nodes), and element i of an [ny][pitch] plane of n elements.
__device__ __forceinline__ uint4 ldg_vec(const uint4* __restrict__ region, long long node,
                                         long long n) {
  return in_range(node, n, OOB_POPS) ? __ldg(region + node) : make_uint4(0u, 0u, 0u, 0u);
}
__device__ __forceinline__ float ldg_plane(const float* __restrict__ p, long long i, long long n) {
  return in_range(i, n, OOB_PLANE) ? __ldg(p + i) : 0.0f;
}
__device__ __forceinline__ void st_plane(float* __restrict__ p, long long i, long long n, float v) {
  if (in_range(i, n, OOB_PLANE)) p[i] = v;
}
// Element i of a plane copied into shared memory asynchronously (cp.async through L1): the
// value is there once the issuing thread has passed cp_async_wait_all() and, for the other
// threads of the block, a barrier after that. An index out of range stores 0 instead.
__device__ __forceinline__ void cp_async_plane(float* sdst, const float* __restrict__ p,
                                               long long i, long long n) {
  if (in_range(i, n, OOB_PLANE)) {
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(sdst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(p + i) : "memory");
  } else {
    *sdst = 0.0f;
  }
}
// The same at a 32-bit index, for indices the host has bounded below 2^31 (the plane index
// y * pitch + x of a grid: lbmice_create refuses larger grids).
__device__ __forceinline__ float ldg_plane(const float* __restrict__ p, int i, long long n) {
  return in_range(i, n, OOB_PLANE) ? __ldg(p + i) : 0.0f;
}
__device__ __forceinline__ void st_plane(float* __restrict__ p, int i, long long n, float v) {
  if (in_range(i, n, OOB_PLANE)) p[i] = v;
}
__device__ __forceinline__ void cp_async_plane(float* sdst, const float* __restrict__ p, int i,
                                               long long n) {
  if (in_range(i, n, OOB_PLANE)) {
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(sdst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(p + i) : "memory");
  } else {
    *sdst = 0.0f;
  }
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;" ::: "memory");
}

// The 9 deviations d_a = p_a - w_a M of one node and lattice from its 16-bit vector v; the
// rest one is d_0 = -sum_{a>0} d_a, since the populations sum to M.
template <class S>
__device__ __forceinline__ void deviations9(uint4 v, float* d) {
  Storage<S>::unpack8(v, d + 1);
  d[0] = -(((d[1] + d[3]) + (d[2] + d[4])) + ((d[5] + d[7]) + (d[6] + d[8])));
}

// Populations of lattice L at a node: stored values for F32, or rebuilt from the moment M
// and the deviations for F16 / BF16.
template <class S>
__device__ __forceinline__ void load9(const typename Storage<S>::T* __restrict__ pops, int L,
                                      long long pstride, long long node, float M, float* out) {
  if (!in_range(node, pstride, OOB_POPS)) {
#pragma unroll
    for (int a = 0; a < 9; ++a) out[a] = 0.0f;
    return;
  }
  if constexpr (Storage<S>::PLANES) {
#pragma unroll
    for (int a = 0; a < 9; ++a) out[a] = __ldg(pops + (9 * L + a) * pstride + node);
  } else if constexpr (!Storage<S>::DEV) {
    if (L == 2) {
      load_lattice_f32(pops + 18 * pstride, pstride, node, out);
    } else {
#pragma unroll
      for (int a = 0; a < 9; ++a) out[a] = __ldg(pops + f32_pop_index(pstride, node, L, a));
    }
  } else {
    decode9<S>(__ldg(reinterpret_cast<const uint4*>(pops + 9 * L * pstride + 8 * node)), M, out);
  }
}

// Store the 9 populations p of lattice L at a node, whose zeroth moment is M (= sum p).
template <class S>
__device__ __forceinline__ void store9(typename Storage<S>::T* __restrict__ pops, int L,
                                       long long pstride, long long node, float M,
                                       const float* p) {
  if (!in_range(node, pstride, OOB_POPS)) return;
  if constexpr (Storage<S>::PLANES) {
#pragma unroll
    for (int a = 0; a < 9; ++a) pops[(9 * L + a) * pstride + node] = p[a];
  } else if constexpr (!Storage<S>::DEV) {
    if (L == 2) {
      store_lattice_f32(pops + 18 * pstride, pstride, node, p);
    } else {
#pragma unroll
      for (int a = 0; a < 9; ++a) pops[f32_pop_index(pstride, node, L, a)] = p[a];
    }
  } else {
    float d[8];
#pragma unroll
    for (int a = 1; a < 9; ++a) d[a - 1] = fmaf(-(a < 5 ? 1.0f / 9.0f : 1.0f / 36.0f), M, p[a]);
    *reinterpret_cast<uint4*>(pops + 9 * L * pstride + 8 * node) = Storage<S>::pack8(d);
  }
}

enum : int { BC_PERIODIC = 0, BC_INLET = 1, BC_OUTLET = 2, BC_FREESLIP = 3 };
enum : int { PLANE_H = 0, PLANE_G = 9, PLANE_F = 18 };

// Lattice constants of one grid, precomputed on the host (lattice units).
struct Consts {
  int nx, ny, pitch;  // pitch: floats per row of a phi array
  int bc[4];
  int stencil;        // gradient stencil (Sec. 3.1.1): 2, 4, 6 or 8
  int fold;           // anisotropy symmetry: 6 (ice, Sec. 2.1) or 4 (validation case)
  int seg_rows;       // rows of the strip segment one march CTA walks (a multiple of 8)
  long long pstride;  // floats between population planes of one node
  long long rstride;  // floats between rows of one population plane
  float Dphi3;       // 3 (W0^2/tau0) dt/dx^2: eta = Dphi3 a_s^2 + 1/2, h^eq flux weight
  float dt_tau0;     // dt/tau0: weight of the phase-field source Q
  float lambda;      // coupling of U into Q
  float Dlat3;       // 3 D dt/dx^2: tau_g = Dlat3 q + 1/2
  float half_Lsat;   // L_sat / 2
  float eps;         // six-fold anisotropy strength
  float kNkeps;      // kappa_N k eps (k = fold): N = kNkeps a_s sin(k theta) (g_y, -g_x)
  float kdrag;       // h nu / (4 (W0/dx)^2): k = kdrag rho (1+phi)^2 (1-phi)
  float inv_tau_f;   // 1 / tau_f
  float guo;         // 1 - 1/(2 tau_f)
  float U_in;        // inlet supersaturation
  float uin_x[4], uin_y[4];  // inlet velocity of each face (inward normal times u_in)
};

// E4 gradient weights (Table 1): shells |c|^2 = 1 and 2.
__device__ constexpr float kW1 = 1.0f / 3.0f;
__device__ constexpr float kW2 = 1.0f / 12.0f;

// Six-fold anisotropy from a lattice gradient (Sec. 2.1): a_s = 1 + eps cos(6 theta) and the
// anisotropic flux N = kappa_N a_s 6 eps sin(6 theta) (g_y, -g_x). cos/sin(6 theta) are the
// real/imaginary parts of (n_x + i n_y)^6 of the unit normal; |g|^2 <= 1e-12 -> isotropic.
template <class T>
__device__ __forceinline__ void aniso(T gx, T gy, T eps, T kNkeps, int fold, T& as, T& Nx,
                                      T& Ny) {
  const T s = gx * gx + gy * gy;
  as = T(1);
  Nx = T(0);
  Ny = T(0);
  if (s > T(1e-12)) {
    const T rinv = T(1) / sqrt(s);
    const T nx = gx * rinv, ny = gy * rinv;
    const T X = nx * nx, Y = ny * ny;
    T cosk, sink;
    if (fold == 4) {  // cos/sin(4 theta) from (n_x + i n_y)^4
      cosk = X * X - T(6) * X * Y + Y * Y;
      sink = T(4) * nx * ny * (X - Y);
    } else {
      cosk = X * X * X - T(15) * X * X * Y + T(15) * X * Y * Y - Y * Y * Y;
      sink = nx * ny * (T(6) * X * X - T(20) * X * Y + T(6) * Y * Y);
    }
    as = T(1) + eps * cosk;
    const T t = kNkeps * as * sink;
    Nx = t * gy;
    Ny = -(t * gx);
  }
}

// Round-to-nearest product and fused multiply-add for float and double: the compiler never
// contracts or reassociates them, so every kernel computing the same expression gets the
// same bits.
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return fma(a, b, c); }

// Packed FP32 pairs (sm_100 family): each operation rounds both lanes to nearest exactly as
// its scalar counterpart would, and issues once for the two lanes.
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 fadd2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 fmul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 pair(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 splat(float a) { return make_float2(a, a); }

// Isotropic gradient with the stencil of the run (Sec. 3.1.1): E2 is the central difference;
// E4, E6, E8 sum w(|c|^2) phi(x + c) c over the neighbour shells of Table 1 with the printed
// weights (they carry the 1/c_s^2). P(dx, dy) is phi at the offset. Every shell is a sum of
// differences of opposite neighbours, grouped so that mirrored fields give exactly mirrored
// gradients, and every product is explicitly rounded.
template <class T, class F>
__device__ __forceinline__ void gradient_stencil(int stencil, F P, T& gx, T& gy) {
  if (stencil == 2) {
    gx = mul_rn(T(0.5), P(1, 0) - P(-1, 0));
    gy = mul_rn(T(0.5), P(0, 1) - P(0, -1));
    return;
  }
  if (stencil == 4) {
    gx = fma_rn(T(1.0 / 3.0), P(1, 0) - P(-1, 0),
                mul_rn(T(1.0 / 12.0), (P(1, 1) - P(-1, 1)) + (P(1, -1) - P(-1, -1))));
    gy = fma_rn(T(1.0 / 3.0), P(0, 1) - P(0, -1),
                mul_rn(T(1.0 / 12.0), (P(1, 1) - P(1, -1)) + (P(-1, 1) - P(-1, -1))));
    return;
  }
  const bool e8 = stencil == 8;
  const T w1 = e8 ? T(4.0 / 21.0) : T(4.0 / 15.0);
  const T w2 = e8 ? T(4.0 / 45.0) : T(1.0 / 10.0);
  const T w4x2 = e8 ? T(2.0 / 60.0) : T(2.0 / 120.0);
  T ax = fma_rn(w1, P(1, 0) - P(-1, 0), mul_rn(w2, (P(1, 1) - P(-1, 1)) + (P(1, -1) - P(-1, -1))));
  T ay = fma_rn(w1, P(0, 1) - P(0, -1), mul_rn(w2, (P(1, 1) - P(1, -1)) + (P(-1, 1) - P(-1, -1))));
  ax = fma_rn(w4x2, P(2, 0) - P(-2, 0), ax);
  ay = fma_rn(w4x2, P(0, 2) - P(0, -2), ay);
  if (e8) {
    const T w5 = T(2.0 / 315.0), w8x2 = T(2.0 / 5040.0);
    // |c|^2 = 5 shell: (1, 2) and (2, 1) families; the factor 2 is exact
    const T dx5 = fma_rn(T(2), (P(2, 1) - P(-2, 1)) + (P(2, -1) - P(-2, -1)),
                         (P(1, 2) - P(-1, 2)) + (P(1, -2) - P(-1, -2)));
    const T dy5 = fma_rn(T(2), (P(1, 2) - P(1, -2)) + (P(-1, 2) - P(-1, -2)),
                         (P(2, 1) - P(2, -1)) + (P(-2, 1) - P(-2, -1)));
    ax = fma_rn(w5, dx5, ax);
    ay = fma_rn(w5, dy5, ay);
    ax = fma_rn(w8x2, (P(2, 2) - P(-2, 2)) + (P(2, -2) - P(-2, -2)), ax);
    ay = fma_rn(w8x2, (P(2, 2) - P(2, -2)) + (P(-2, 2) - P(-2, -2)), ay);
  }
  gx = ax;
  gy = ay;
}

// Ghost resolution of one axis for phi reads (R: periodic wrap, zero-gradient clamp,
// free-slip reflection about the wall half a cell out, inlet = vapour). Returns false for
// an inlet ghost. Valid for coordinates up to a grid length outside.
__device__ __forceinline__ bool axis_phi(int v, int n, int bc_lo, int bc_hi, int& out) {
  if (v < 0) {
    if (bc_lo == BC_PERIODIC) { out = v + n; return true; }
    if (bc_lo == BC_OUTLET) { out = 0; return true; }
    if (bc_lo == BC_FREESLIP) { out = -1 - v; return true; }
    return false;
  }
  if (v >= n) {
    if (bc_hi == BC_PERIODIC) { out = v - n; return true; }
    if (bc_hi == BC_OUTLET) { out = n - 1; return true; }
    if (bc_hi == BC_FREESLIP) { out = 2 * n - 1 - v; return true; }
    return false;
  }
  out = v;
  return true;
}

}  // namespace lbmice
