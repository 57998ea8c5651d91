// The fused collide-stream step: one launch advances h, g and f by one time step
// (arXiv 2101.07163, Sec. 2.2.1-2.2.3) over the whole grid.
//
// Every kernel here works in three phases per group of destination nodes:
//   A. phi^n around the group (ghosts resolved) -> shared memory, while each thread's own
//      populations are loaded into registers;
//   B. every source node the group pulls from is collided once: moments, the gradient of phi
//      from the shared tile, a_s and the anisotropic flux, the drag, and the 27 post-collision
//      populations, which go to shared memory (h already divided by a_s^2 and paired with g,
//      plus B = 1 - 1/a_s^2, so the pull of Eq. (d) is one FMA);
//   C. each destination pulls its 27 populations from shared memory, applies Eq. (d), and
//      writes h, g, f and phi^{n+1} = sum h to HBM.
// Two ways of grouping the destinations:
//   - march_kernel (the default E4 six-fold scheme): a CTA of 8 warps walks up a segment of a
//     strip of 32 columns, 8 rows per pass; warp w collides the 32 nodes of one row and pulls
//     the 30 inner ones. Rows collided in one pass stay in a ring of shared rows for the next,
//     so the only nodes collided twice are the strip's two edge columns (1/15 of the work)
//     and two rows where a segment starts.
//   - step_kernel: one CTA per TX x TY tile, which collides its tile plus a one-node ring
//     (used for the wider stencils, and as alternative shapes of the batched launch).
// HBM traffic per node: 27 populations in and out, phi^n, phi^{n-1} in, phi^{n+1} out; the
// re-read edge columns and rows hit L2.
#pragma once

#include <type_traits>

#include "../../include/lbmice.h"
#include "lbmice_device.cuh"
#include "lbmice_tma.cuh"

namespace lbmice {

struct StepPtrs {
  const void* pin;                    // populations at time n (storage type of the kernel)
  void* pout;                         // populations at time n + 1
  const float* __restrict__ phi_n;    // phi^n (the zeroth moment of h)
  const float* __restrict__ phi_nm1;  // phi^{n-1}
  float* __restrict__ phi_np1;        // phi^{n+1}
  const float* __restrict__ U_n;      // 16-bit storage only: U^n, rho^n and their updates
  float* __restrict__ U_np1;
  const float* __restrict__ rho_n;
  float* __restrict__ rho_np1;
  // tensor maps of this step's inputs (in device memory), six per step: 16-bit storage's L2
  // prefetch boxes (deviation vectors, U^n, rho^n, unused, phi^{n-1}; unset for FP32) and
  // phi^n in the march's phi-ring blocks (slot 5). Null (buffers without maps): no
  // prefetch, and the phi ring is filled by cp.async.
  const CUtensorMap* tm;
  // pin and pout as kRegions region bases, precomputed on the host (step_regions), so that
  // every population access of a step is a 32-bit node index (node < pstride < 2^31) on a
  // kernel-parameter base. FP32: the (h,g) quads of directions 1-2, 3-4, 5-6, 7-8 (float4),
  // the (h_0,g_0) pairs (float2), the f quads 1-4 and 5-8 (float4) and f_0 (float); 16-bit:
  // the h, g and f deviation vectors (uint4).
  const void* rin[8];
  void* rout[8];
};
constexpr int kRegions = 8;

// Prefetch the line holding p into L1 (an address inside a buffer; nothing to wait for).
__device__ __forceinline__ void prefetch_l1(const void* p) {
  asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

// ---- population accesses of a step through the region bases --------------------------------
__device__ __forceinline__ void load_hg_rg(const Consts& C, const StepPtrs& P, int node,
                                           float2* hg) {
  if (!in_range(node, C.pstride, OOB_POPS)) {
#pragma unroll
    for (int a = 0; a < 9; ++a) hg[a] = make_float2(0.0f, 0.0f);
    return;
  }
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const float4 v = __ldg(static_cast<const float4*>(P.rin[p]) + node);
    hg[2 * p + 1] = make_float2(v.x, v.y);
    hg[2 * p + 2] = make_float2(v.z, v.w);
  }
  hg[0] = __ldg(static_cast<const float2*>(P.rin[4]) + node);
}
__device__ __forceinline__ void store_hg_rg(const Consts& C, const StepPtrs& P, int node,
                                            const float2* hg) {
  if (!in_range(node, C.pstride, OOB_POPS)) return;
#pragma unroll
  for (int p = 0; p < 4; ++p)
    static_cast<float4*>(P.rout[p])[node] =
        make_float4(hg[2 * p + 1].x, hg[2 * p + 1].y, hg[2 * p + 2].x, hg[2 * p + 2].y);
  static_cast<float2*>(P.rout[4])[node] = hg[0];
}
__device__ __forceinline__ void load_f_rg(const Consts& C, const StepPtrs& P, int node, float* f) {
  if (!in_range(node, C.pstride, OOB_POPS)) {
#pragma unroll
    for (int a = 0; a < 9; ++a) f[a] = 0.0f;
    return;
  }
  const float4 p = __ldg(static_cast<const float4*>(P.rin[5]) + node);
  const float4 q = __ldg(static_cast<const float4*>(P.rin[6]) + node);
  f[0] = __ldg(static_cast<const float*>(P.rin[7]) + node);
  f[1] = p.x;
  f[2] = p.y;
  f[3] = p.z;
  f[4] = p.w;
  f[5] = q.x;
  f[6] = q.y;
  f[7] = q.z;
  f[8] = q.w;
}
__device__ __forceinline__ void store_f_rg(const Consts& C, const StepPtrs& P, int node,
                                           const float* f) {
  if (!in_range(node, C.pstride, OOB_POPS)) return;
  static_cast<float4*>(P.rout[5])[node] = make_float4(f[1], f[2], f[3], f[4]);
  static_cast<float4*>(P.rout[6])[node] = make_float4(f[5], f[6], f[7], f[8]);
  static_cast<float*>(P.rout[7])[node] = f[0];
}
// 16-bit: the deviation vector of lattice L (0 h, 1 g, 2 f) at a node.
__device__ __forceinline__ uint4 ldg_vec_rg(const Consts& C, const StepPtrs& P, int L, int node) {
  return in_range(node, C.pstride, OOB_POPS) ? __ldg(static_cast<const uint4*>(P.rin[L]) + node)
                                             : make_uint4(0u, 0u, 0u, 0u);
}
__device__ __forceinline__ void stg_vec_rg(const Consts& C, const StepPtrs& P, int L, int node,
                                           uint4 v) {
  if (in_range(node, C.pstride, OOB_POPS)) static_cast<uint4*>(P.rout[L])[node] = v;
}

// Collided populations of SN source nodes in shared memory: (h*_a / a_s^2, g*_a) pairs,
// f*_a, and B = 1 - 1/a_s^2 of every source node.
struct PostTile {
  float2* hg;  // [9][SN]
  float* f;    // [9][SN] (flow only)
  float* B;    // [SN]
  int SN;
  template <bool FLOW>
  __host__ __device__ static constexpr size_t floats(int SN) { return (size_t)SN * (FLOW ? 28 : 19); }
  template <bool FLOW>
  __device__ static PostTile at(float* base, int SN) {
    PostTile T;
    T.hg = reinterpret_cast<float2*>(base);
    T.f = base + 18 * SN;
    T.B = T.f + (FLOW ? 9 * SN : 0);
    T.SN = SN;
    return T;
  }
};

// Tile of TX x TY destination nodes for a gradient stencil of radius R (1: the default E4
// with six-fold anisotropy, specialised; 2: any stencil up to E8 and either fold): the phi
// tile has a halo of R + 1 (the stencil around every ring node), the collided source tile a
// halo of 1.
template <int TX, int TY, int R = 1>
struct Tile {
  static constexpr int H = R + 1;
  static constexpr int PW = TX + 2 * H;              // phi tile row
  static constexpr int PN = PW * (TY + 2 * H);
  static constexpr int SW = TX + 2;                  // source tile row (halo 1)
  static constexpr int SN = SW * (TY + 2);
  static constexpr int NRING = SN - TX * TY;
  static constexpr int NT = TX * TY;
  template <bool FLOW>
  static constexpr size_t smem_bytes() {
    return sizeof(float) * (PostTile::floats<FLOW>(SN) + PN);
  }
};

// phi around the node a collision is taken at, in the 2D tile: v(dx, dy) = phi at the
// offset; pc is the centre's index in the tile.
struct TileView {
  const float* s;
  int pc, PW, PN, R;
  __device__ __forceinline__ float operator()(int dx, int dy) const { return s[pc + dy * PW + dx]; }
  __device__ __forceinline__ bool ok() const {
    return in_range(pc - R * (PW + 1), PN, OOB_SHARED) && in_range(pc + R * (PW + 1), PN, OOB_SHARED);
  }
};

// The loads of a thread's own node (inside the grid), issued before the phi tile's barrier so
// that their latency overlaps the tile's: FP32 keeps the populations, 16-bit storage the
// raw deviation vectors and the moments U, rho (phi comes from the tile).
template <class S, bool FLOW, bool DEV = Storage<S>::DEV>
struct OwnIn;
template <class S, bool FLOW>
struct OwnIn<S, FLOW, false> {
  bool valid;
  float2 hg[9];
  float f[9], php;
};
template <class S, bool FLOW>
struct OwnIn<S, FLOW, true> {
  bool valid;
  uint4 h, g, f;
  float U, rho, php;
};

template <class S, bool FLOW>
__device__ __forceinline__ void own_load(const Consts& C, const StepPtrs& P, int X, int Y,
                                         OwnIn<S, FLOW>& in) {
  using ST = Storage<S>;
  in.valid = X >= 0 && Y >= 0 && X < C.nx && Y < C.ny;
  if (!in.valid) return;
  const int idx = Y * C.pitch + X;
  const int nd = Y * (int)C.rstride + X;
  const long long np = (long long)C.pitch * C.ny;
  if constexpr (!ST::DEV) {
    load_hg_rg(C, P, nd, in.hg);
    if (FLOW) load_f_rg(C, P, nd, in.f);
  } else {
    in.h = ldg_vec_rg(C, P, 0, nd);
    in.g = ldg_vec_rg(C, P, 1, nd);
    in.U = ldg_plane(P.U_n, idx, np);
    if (FLOW) {
      in.f = ldg_vec_rg(C, P, 2, nd);
      in.rho = ldg_plane(P.rho_n, idx, np);
    }
  }
  in.php = ldg_plane(P.phi_nm1, idx, np);
}

// ---- L2 prefetch of a march pass -----------------------------------------------------------
// With 16-bit storage the populations a march pass collides (rows y .. y + 7, columns
// X0 - 1 .. X0 + 30) are prefetched into L2 by TMA a pass ahead, one box per stored plane
// group, so that the pass's own loads hit L2: the deviation vectors [3][8][32 x 8 halves],
// U, rho and phi^{n-1} [8][36 from column xa], xa = (X0 - 1) rounded down to a multiple of 4,
// so that every box starts on a 16-byte boundary (parts outside the grid are skipped).
// Tensor map slots (StepPtrs::tm): vectors, U, rho, (unused), phi^{n-1}; slot 5 is the phi^n
// map of the phi ring. FP32 steps, bandwidth-bound, run the plain march and prefetch nothing.
// Thread 0: prefetch into L2 the boxes of the pass whose collided rows start at row y.
template <bool FLOW, class S>
__device__ __forceinline__ void prefetch_issue(const StepPtrs& P, int X0, int y) {
  if constexpr (Storage<S>::DEV) {
    const int xa = (X0 - 1) & ~3;
    tma_prefetch_3d(P.tm + 0, 8 * (X0 - 1), y, 0);
    tma_prefetch_2d(P.tm + 1, xa, y);
    if (FLOW) tma_prefetch_2d(P.tm + 2, xa, y);
    tma_prefetch_2d(P.tm + 4, xa, y);
  }
}

// Deviations (d^h_a, d^g_a) of a node from its two 16-bit vectors; the rest pair is minus the
// sum of the others (summed in the pairing of sum9).
template <class S>
__device__ __forceinline__ void deviations_hg(uint4 vh, uint4 vg, float2* hg) {
  float dh[8], dg[8];
  Storage<S>::unpack8(vh, dh);
  Storage<S>::unpack8(vg, dg);
#pragma unroll
  for (int a = 1; a < 9; ++a) hg[a] = pair(dh[a - 1], dg[a - 1]);
  const float2 s = fadd2(fadd2(fadd2(hg[1], hg[3]), fadd2(hg[2], hg[4])),
                         fadd2(fadd2(hg[5], hg[7]), fadd2(hg[6], hg[8])));
  hg[0] = pair(-s.x, -s.y);
}

// sum9 of pairs, lane by lane, in the same grouping as sum9.
__device__ __forceinline__ float2 sum9_2(const float2* v) {
  return fadd2(v[0], fadd2(fadd2(fadd2(v[1], v[3]), fadd2(v[2], v[4])),
                           fadd2(fadd2(v[5], v[7]), fadd2(v[6], v[8]))));
}

// Collide the source node at global coordinates (X, Y) in [-1, nx] x [-1, ny] and store its
// post-collision populations in slot `node` of the shared tile T. view_at(sx, sy) returns the
// phi view (operator()(dx, dy), ok()) centred on the tile position of this node shifted by
// (sx, sy): a ghost node of a non-periodic face takes the collision of the interior node its
// face rule maps it to (directions mirrored across a free-slip wall), or the fixed inlet
// state. OWN: the node is the thread's destination; its pre-collision h (as populations) goes
// to hown, for the pull of Eq. (d), and its loads may come from pre.
//
// The collision, Sec. 2.2.1-2.2.3, is evaluated in a factored form with per-node
// coefficients (every product and sum an explicit round-to-nearest operation, so every kernel
// that collides a node produces the same bits):
//   phase field, Eq. (d)/(e): h* = h - (h - h^eq)/eta + w Q dt/tau0, h^eq = w (phi - 3 Dphi
//     c.N), stored divided by a_s^2:  h*/a_s^2 = a1 h + w (a2 - a3 c.N);
//   vapour: g* = g - (g - g^eq)/tau_g + w S dt, g^eq = w U (1 + 3 c.u*):
//     g* = b1 g + w (b2 + b3 c.u*);
//   flow: BGK to the second-order f^eq(rho, u*) plus Guo forcing of F = -k u*; since c.F =
//     -k c.u*, f* = c1 f + w (c2 + c3 c.u* + c4 (c.u*)^2) with
//     c2 = r (1 - 3/2 u*.u*) + 3 gamma k u*.u*, c3 = 3 (r - gamma k), c4 = 9/2 (r - 2 gamma k),
//     r = rho / tau_f, gamma = 1 - 1/(2 tau_f).
// The projections c.v are sums and exact negations (cdot), so mirror images of a state stay
// bit-exact mirror images. (h*_a/a_s^2, g*_a) go to shared memory as one pair.
template <bool FLOW, class S, bool OWN, int R, class ViewAt, bool GHOSTS = true>
__device__ __forceinline__ void collide_source(const Consts& C, const StepPtrs& P, int X, int Y,
                                               int node, const ViewAt& view_at,
                                               const PostTile& T, float* hown,
                                               const OwnIn<S, FLOW>* pre = nullptr) {
  if (!in_range(node, T.SN, OOB_SHARED)) return;
  int mx = X, my = Y, shx = 0, shy = 0;
  bool mirx = false, miry = false;
  int inlet = -1;
  // !GHOSTS: the caller knows (X, Y) is inside the grid
  if (GHOSTS && (X < 0 || X >= C.nx)) {
    const int face = X < 0 ? 0 : 1;
    const int bc = X < 0 ? C.bc[0] : C.bc[1];
    if (bc == BC_PERIODIC) {
      mx = X < 0 ? X + C.nx : X - C.nx;
    } else {
      mx = X < 0 ? 0 : C.nx - 1;
      shx = X < 0 ? 1 : -1;
      mirx = bc == BC_FREESLIP;
      if (bc == BC_INLET) inlet = face;
    }
  }
  if (GHOSTS && (Y < 0 || Y >= C.ny)) {
    const int face = Y < 0 ? 2 : 3;
    const int bc = Y < 0 ? C.bc[2] : C.bc[3];
    if (bc == BC_PERIODIC) {
      my = Y < 0 ? Y + C.ny : Y - C.ny;
    } else {
      my = Y < 0 ? 0 : C.ny - 1;
      shy = Y < 0 ? 1 : -1;
      miry = bc == BC_FREESLIP;
      if (bc == BC_INLET && inlet < 0) inlet = face;
    }
  }
  using ST = Storage<S>;
  const int idx = my * C.pitch + mx;  // < 2^31: lbmice_create refuses larger grids
  const int nd = my * (int)C.rstride + mx;
  const int SN = T.SN;

  if (GHOSTS && inlet >= 0) {
    // Inlet ghost: vapour at the inlet state, flow equilibrium at the adjacent density.
    const float ux = inlet == 0 ? C.uin_x[0] : inlet == 1 ? C.uin_x[1]
                   : inlet == 2 ? C.uin_x[2] : C.uin_x[3];
    const float uy = inlet == 0 ? C.uin_y[0] : inlet == 1 ? C.uin_y[1]
                   : inlet == 2 ? C.uin_y[2] : C.uin_y[3];
    float rho = 1.0f;
    if (FLOW) {
      if constexpr (ST::DEV) {
        rho = ldg_plane(P.rho_n, idx, (long long)C.pitch * C.ny);
      } else {
        float fv[9];
        load_f_rg(C, P, nd, fv);
        rho = sum9(fv);
      }
    }
    const float uu = ux * ux + uy * uy;
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      const float cu = cdot(a, ux, uy);
      T.hg[a * SN + node] = pair(-w_of(a), w_of(a) * C.U_in * (1.0f + 3.0f * cu));
      if (FLOW) T.f[a * SN + node] = w_of(a) * rho * (1.0f + 3.0f * cu + 4.5f * cu * cu - 1.5f * uu);
    }
    T.B[node] = 0.0f;
    return;
  }

  const auto V = view_at(shx, shy);
  if (!V.ok()) return;
  // ---- populations and moments at time n (Sec. 2.2) ----
  const float ph = V(0, 0);
  // FP32: the populations. 16-bit: their deviations d_a = p_a - w_a M from the stored
  // moments M (phi, U, rho), with d_0 = -sum_{a>0} d_a; the moments are the stored ones and
  // the momentum is sum c_a d_a (the w_a M terms cancel exactly).
  float2 hg[9];
  float fv[9];
  float php, U, rho = 1.0f;
  if (OWN && pre && pre->valid) {  // loaded before the phi tile's barrier
    if constexpr (!ST::DEV) {
#pragma unroll
      for (int a = 0; a < 9; ++a) {
        hg[a] = pre->hg[a];
        if (FLOW) fv[a] = pre->f[a];
      }
    } else {
      deviations_hg<S>(pre->h, pre->g, hg);
      U = pre->U;
      if (FLOW) {
        deviations9<S>(pre->f, fv);
        rho = pre->rho;
      }
    }
    php = pre->php;
  } else {
    if constexpr (!ST::DEV) {
      load_hg_rg(C, P, nd, hg);
      if (FLOW) load_f_rg(C, P, nd, fv);
    } else {
      const long long np = (long long)C.pitch * C.ny;
      deviations_hg<S>(ldg_vec_rg(C, P, 0, nd), ldg_vec_rg(C, P, 1, nd), hg);
      U = ldg_plane(P.U_n, idx, np);
      if (FLOW) {
        deviations9<S>(ldg_vec_rg(C, P, 2, nd), fv);
        rho = ldg_plane(P.rho_n, idx, np);
      }
    }
    php = ldg_plane(P.phi_nm1, idx, (long long)C.pitch * C.ny);
  }
  if constexpr (!ST::DEV) {
    U = hg[0].y + (((hg[1].y + hg[3].y) + (hg[2].y + hg[4].y)) +
                   ((hg[5].y + hg[7].y) + (hg[6].y + hg[8].y)));
    if (FLOW) rho = sum9(fv);
  }
  float jx = 0.0f, jy = 0.0f;
  if (FLOW) {
    jx = sumcx9(fv);
    jy = sumcy9(fv);
  }

  // ---- gradient of phi (Sec. 3.1.1, Table 1) and anisotropy (Sec. 2.1) ----
  float gx, gy;
  if constexpr (R == 1) {  // E4 with six-fold anisotropy: the default, with no run-time variant branch
    const float pE = V(1, 0), pW = V(-1, 0), pN = V(0, 1), pS = V(0, -1);
    const float pNE = V(1, 1), pNW = V(-1, 1), pSE = V(1, -1), pSW = V(-1, -1);
    gx = fmaf(kW1, pE - pW, __fmul_rn(kW2, (pNE - pNW) + (pSE - pSW)));
    gy = fmaf(kW1, pN - pS, __fmul_rn(kW2, (pNE - pSE) + (pNW - pSW)));
  } else {  // any stencil and fold, chosen at run time, on a phi tile of halo R + 1 = 3
    gradient_stencil<float>(C.stencil, V, gx, gy);
  }
  // Every product and sum from here to the collision is an explicit fmaf or round-to-nearest
  // operation, like the collision itself: no kernel that collides a node may contract them
  // differently, so single-grid and batched kernels give the same bits.
  float as = 1.0f, Nx = 0.0f, Ny = 0.0f;
  {
    const float s2 = fmaf(gx, gx, __fmul_rn(gy, gy));
    if (s2 > 1e-12f) {  // |grad phi|^2 <= 1e-12: isotropic, no anisotropic flux
      const float rinv = rsqrtf(s2);
      const float nx = __fmul_rn(gx, rinv), ny = __fmul_rn(gy, rinv);
      const float X2 = __fmul_rn(nx, nx), Y2 = __fmul_rn(ny, ny);
      const float XX = __fmul_rn(X2, X2), YY = __fmul_rn(Y2, Y2), XY = __fmul_rn(X2, Y2);
      const float nxny = __fmul_rn(nx, ny);
      float cosk, sink;
      if (R != 1 && C.fold == 4) {  // the four-fold validation case: cos/sin(4 theta)
        cosk = fmaf(-6.0f, XY, XX + YY);                       // X^2 - 6XY + Y^2
        sink = __fmul_rn(__fmul_rn(4.0f, nxny), X2 - Y2);      // 4 nx ny (X - Y)
      } else {  // six-fold (ice): cos/sin(6 theta)
        cosk = __fmul_rn(X2 - Y2, fmaf(-14.0f, XY, XX + YY));  // X^3 - 15X^2Y + 15XY^2 - Y^3
        sink = __fmul_rn(nxny, fmaf(-20.0f, XY, __fmul_rn(6.0f, XX + YY)));
      }
      as = fmaf(C.eps, cosk, 1.0f);
      const float t = __fmul_rn(__fmul_rn(C.kNkeps, as), sink);
      Nx = __fmul_rn(t, gy);
      Ny = -__fmul_rn(t, gx);
    }
  }
  const float as2 = __fmul_rn(as, as);
  const float inv_as2 = __fdividef(1.0f, as2);
  const float inv_eta = __fdividef(1.0f, fmaf(C.Dphi3, as2, 0.5f));
  const float omp2 = fmaf(-ph, ph, 1.0f);
  const float srcQ =
      __fmul_rn((ph - __fmul_rn(__fmul_rn(ph, ph), ph)) +
                    __fmul_rn(__fmul_rn(C.lambda, U), __fmul_rn(omp2, omp2)),
                C.dt_tau0);

  // ---- flow velocity with solid damping (Sec. 2.2.1) ----
  float usx = 0.0f, usy = 0.0f, k = 0.0f;
  if (FLOW) {
    const float onep = 1.0f + ph;
    k = __fmul_rn(__fmul_rn(__fmul_rn(C.kdrag, rho), __fmul_rn(onep, onep)), 1.0f - ph);
    const float inv = __fdividef(1.0f, fmaf(0.5f, k, rho));
    const float sfac = __fmul_rn(0.5f, 1.0f - ph);
    usx = __fmul_rn(sfac, __fmul_rn(jx, inv));
    usy = __fmul_rn(sfac, __fmul_rn(jy, inv));
  }
  // ---- vapour relaxation and source (Sec. 2.2.2) ----
  const float q = fminf(fmaxf(1.0f - ph, 0.0f), 2.0f);
  const float inv_tg = __fdividef(1.0f, fmaf(C.Dlat3, q, 0.5f));
  const float srcU = __fmul_rn(-C.half_Lsat, ph - php);

  if (OWN) {  // the own node's h populations, for the pull of Eq. (d)
#pragma unroll
    for (int a = 0; a < 9; ++a) hown[a] = ST::DEV ? fmaf(w_of(a), ph, hg[a].x) : hg[a].x;
  }

  // ---- the collision (factored) ----
  const float a1 = __fmul_rn(1.0f - inv_eta, inv_as2);
  float a2 = __fmul_rn(fmaf(ph, inv_eta, srcQ), inv_as2);
  const float a3 = __fmul_rn(__fmul_rn(C.Dphi3, inv_eta), inv_as2);
  const float b1 = 1.0f - inv_tg;
  float b2 = fmaf(U, inv_tg, srcU);
  const float b3 = __fmul_rn(__fmul_rn(3.0f, U), inv_tg);
  if (ST::DEV) {  // deviations: each collision is affine in p_a, slope a1 (b1) times M moves
    a2 = fmaf(a1, ph, a2);  // into the constant term
    b2 = fmaf(b1, U, b2);
  }
  float c1 = 0.0f, c2 = 0.0f, c3 = 0.0f, c4 = 0.0f;
  if (FLOW) {
    c1 = 1.0f - C.inv_tau_f;
    const float r = __fmul_rn(rho, C.inv_tau_f);
    const float uu = fmaf(usx, usx, __fmul_rn(usy, usy));
    const float gk = __fmul_rn(C.guo, k);
    c2 = fmaf(r, fmaf(-1.5f, uu, 1.0f), __fmul_rn(__fmul_rn(3.0f, gk), uu));
    if (ST::DEV) c2 = fmaf(c1, rho, c2);
    c3 = __fmul_rn(3.0f, r - gk);
    c4 = __fmul_rn(4.5f, fmaf(-2.0f, gk, r));
  }
  // Each collided value is stored as it is formed (nothing staged: the kernels stay within
  // their register budgets); behind a free-slip wall the directions are mirrored, a uniform
  // branch, so the common path stores at fixed shared-memory offsets.
  const auto form = [&](auto mirrored) {
    constexpr bool M = decltype(mirrored)::value;
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      int am = a;
      if constexpr (M) {
        am = mirx ? mirx_of(a) : a;
        am = miry ? miry_of(am) : am;
      }
      const int slot = am * SN + node;
      if (a == 0) {  // c_0 = 0: the projection terms vanish exactly (fmaf(x, 0, y) = y)
        T.hg[slot] = pair(fmaf(hg[0].x, a1, __fmul_rn(w_of(0), a2)),
                          fmaf(hg[0].y, b1, __fmul_rn(w_of(0), b2)));
        if (FLOW) T.f[slot] = fmaf(fv[0], c1, __fmul_rn(w_of(0), c2));
        continue;
      }
      T.hg[slot] = pair(fmaf(hg[a].x, a1, __fmul_rn(w_of(a), fmaf(-a3, cdot(a, Nx, Ny), a2))),
                        fmaf(hg[a].y, b1, __fmul_rn(w_of(a), fmaf(b3, cdot(a, usx, usy), b2))));
      if (FLOW) {
        const float cu = cdot(a, usx, usy);
        T.f[slot] = fmaf(fv[a], c1, __fmul_rn(w_of(a), fmaf(fmaf(c4, cu, c3), cu, c2)));
      }
    }
  };
  if (GHOSTS && (mirx || miry)) form(std::true_type{}); else form(std::false_type{});
  T.B[node] = 1.0f - inv_as2;
}

// The pull of destination (X, Y), Eq. (d) for h: src(a) is the shared slot of the source node
// y - c_a; writes h, g, f and phi^{n+1} (16-bit storage: U^{n+1}, rho^{n+1} too).
template <bool FLOW, class S, class SrcOf>
__device__ __forceinline__ void pull_store(const Consts& C, const StepPtrs& P, int X, int Y,
                                           const SrcOf& src, const PostTile& T,
                                           const float* hown) {
  using ST = Storage<S>;
  const int SN = T.SN;
  const int idx = Y * C.pitch + X;
  const long long np = (long long)C.pitch * C.ny;
  const int nd = Y * (int)C.rstride + X;
  float2 hg[9];
  float fn[9];
#pragma unroll
  for (int a = 0; a < 9; ++a) {
    const int s = src(a);
    float2 v = T.hg[a * SN + s];
    v.x = fmaf(hown[a], T.B[s], v.x);
    hg[a] = v;
    if (FLOW) fn[a] = T.f[a * SN + s];
  }
  if constexpr (!ST::DEV) {
    store_hg_rg(C, P, nd, hg);
    if (FLOW) store_f_rg(C, P, nd, fn);
    const float phin = hg[0].x + (((hg[1].x + hg[3].x) + (hg[2].x + hg[4].x)) +
                                  ((hg[5].x + hg[7].x) + (hg[6].x + hg[8].x)));
    st_plane(P.phi_np1, idx, np, phin);
  } else {
    // 16-bit storage: the moments of the pulled populations are stored in FP32 and the
    // moving populations as deviations d_a = p_a - w_a M from them
    const float2 m = sum9_2(hg);  // (phi^{n+1}, U^{n+1})
    st_plane(P.phi_np1, idx, np, m.x);
    st_plane(P.U_np1, idx, np, m.y);
    float dh[8], dg[8];
#pragma unroll
    for (int a = 1; a < 9; ++a) {
      const float2 d = ffma2(splat(-w_of(a)), m, hg[a]);
      dh[a - 1] = d.x;
      dg[a - 1] = d.y;
    }
    stg_vec_rg(C, P, 0, nd, ST::pack8(dh));
    stg_vec_rg(C, P, 1, nd, ST::pack8(dg));
    if (FLOW) {
      const float rn = sum9(fn);
      st_plane(P.rho_np1, idx, np, rn);
      float df[8];
#pragma unroll
      for (int a = 1; a < 9; a += 2) {
        const float2 d = ffma2(splat(-w_of(a)), splat(rn), pair(fn[a], fn[a + 1]));
        df[a - 1] = d.x;
        df[a] = d.y;
      }
      stg_vec_rg(C, P, 2, nd, ST::pack8(df));
    }
  }
}

// phi^n of a tile with origin (x0, y0) and a halo of H nodes into sphi (PW x PH values),
// ghosts resolved (beyond the grid's halo of R: 0, never read).
template <int PW, int PH>
__device__ __forceinline__ void load_phi_tile(const Consts& C, const StepPtrs& P, int x0, int y0,
                                              int H, int R, float* sphi, int tid, int nthreads) {
  constexpr int PN = PW * PH;
  if (x0 >= H && y0 >= H && x0 - H + PW <= C.nx && y0 - H + PH <= C.ny) {
    // the halo lies inside the grid (almost every tile): no ghost resolution
    const float* __restrict__ pb = P.phi_n + (long long)(y0 - H) * C.pitch + (x0 - H);
    const int pitch = (int)C.pitch;
    for (int i = tid; i < PN; i += nthreads) {
      const int lx = i % PW, ly = i / PW;
      if (in_range((long long)(y0 - H + ly) * C.pitch + (x0 - H + lx),
                   (long long)C.pitch * C.ny, OOB_PLANE))
        sphi[i] = __ldg(pb + ly * pitch + lx);
    }
    return;
  }
  for (int i = tid; i < PN; i += nthreads) {
    const int lx = i % PW, ly = i / PW;
    const int X = x0 - H + lx, Y = y0 - H + ly;
    int gx, gy;
    float v = -1.0f;
    if (X > C.nx + R || Y > C.ny + R) {
      v = 0.0f;  // beyond the grid's halo (ragged last tile): never read
    } else if (axis_phi(X, C.nx, C.bc[0], C.bc[1], gx) &&
               axis_phi(Y, C.ny, C.bc[2], C.bc[3], gy)) {
      v = ldg_plane(P.phi_n, (long long)gy * C.pitch + gx, (long long)C.pitch * C.ny);
    }
    sphi[i] = v;
  }
}

// One TX x TY tile with origin (x0, y0), computed by the TX * TY threads of the CTA (thread
// tid owns node (x0 + tid % TX, y0 + tid / TX)). smem holds Tile<TX, TY, R>::smem_bytes.
// PRE: issue the own node's loads before the phi tile's barrier (OwnIn).
template <int TX, int TY, bool FLOW, class S, int R = 1, bool PRE = true>
__device__ __forceinline__ void step_tile(const Consts& C, const StepPtrs& P, int x0, int y0,
                                          float* smem) {
  using T = Tile<TX, TY, R>;
  const PostTile post = PostTile::at<FLOW>(smem, T::SN);
  float* sphi = smem + PostTile::floats<FLOW>(T::SN);
  const int tid = threadIdx.x;
  const int tx = tid % TX, ty = tid / TX;

  // the own node's populations, in flight while the phi tile loads
  OwnIn<S, FLOW> own;
  if (PRE) own_load<S, FLOW>(C, P, x0 + tx, y0 + ty, own);
  else own.valid = false;

  // ---- A: phi^n with a halo of H = R + 1 nodes ----
  load_phi_tile<T::PW, TY + 2 * T::H>(C, P, x0, y0, T::H, R, sphi, tid, T::NT);
  __syncthreads();

  // ---- B: collide the tile (own node per thread) and its one-node ring ----
  float hown[9];
  auto view_of = [&](int sx, int sy) {
    return [=](int shx, int shy) {
      return TileView{sphi, (sy + shy + R) * T::PW + (sx + shx + R), T::PW, T::PN, R};
    };
  };
  {
    const int X = x0 + tx, Y = y0 + ty;
    if (X <= C.nx && Y <= C.ny)
      collide_source<FLOW, S, true, R>(C, P, X, Y, (ty + 1) * T::SW + tx + 1,
                                       view_of(tx + 1, ty + 1), post, hown, &own);
  }
  for (int r = tid; r < T::NRING; r += T::NT) {
    // ring order: bottom row, top row, then left and right columns
    int sx, sy;
    if (r < T::SW) { sx = r; sy = 0; }
    else if (r < 2 * T::SW) { sx = r - T::SW; sy = TY + 1; }
    else { const int k = r - 2 * T::SW; sy = 1 + (k >> 1); sx = (k & 1) ? TX + 1 : 0; }
    const int X = x0 - 1 + sx, Y = y0 - 1 + sy;
    if (X >= -1 && X <= C.nx && Y >= -1 && Y <= C.ny)
      collide_source<FLOW, S, false, R>(C, P, X, Y, sy * T::SW + sx, view_of(sx, sy), post,
                                        nullptr);
  }
  __syncthreads();

  // ---- C: pull, Eq. (d) for h, write populations and phi^{n+1} ----
  const int X = x0 + tx, Y = y0 + ty;
  if (X >= C.nx || Y >= C.ny) return;  // (this thread has no node in this tile)
  // the nine pull sources span tile positions ty..ty+2 x tx..tx+2
  if (!in_range(ty * T::SW + tx, T::SN, OOB_SHARED) ||
      !in_range((ty + 2) * T::SW + tx + 2, T::SN, OOB_SHARED))
    return;
  pull_store<FLOW, S>(C, P, X, Y,
                      [&](int a) { return (ty + 1 - cy_of(a)) * T::SW + (tx + 1 - cx_of(a)); },
                      post, hown);
}

// One CTA per TX x TY tile. FP32 storage is held to 64 registers (4 CTAs of 256 threads per
// SM); the 16-bit forms keep the compiler's own allocation.
template <int TX, int TY, bool FLOW, class S, int R>
__global__ std::enable_if_t<!Storage<S>::DEV> __launch_bounds__(TX* TY, 4)
    step_kernel(const Consts C, const StepPtrs P) {
  extern __shared__ __align__(16) float smem[];
  step_tile<TX, TY, FLOW, S, R>(C, P, blockIdx.x * TX, blockIdx.y * TY, smem);
}
template <int TX, int TY, bool FLOW, class S, int R>
__global__ std::enable_if_t<Storage<S>::DEV> __launch_bounds__(TX* TY)
    step_kernel(const Consts C, const StepPtrs P) {
  extern __shared__ __align__(16) float smem[];
  step_tile<TX, TY, FLOW, S, R>(C, P, blockIdx.x * TX, blockIdx.y * TY, smem);
}

// ---- the column march (default scheme) ---------------------------------------------------
// CTA of kMarchRows warps; warp w handles one row of a 32-column strip per pass. A strip of
// grid columns [X0, X0 + 30) is collided over columns X0 - 1 .. X0 + 30 (lane l: X0 - 1 + l)
// and pulled over lanes 1..30.
constexpr int kMarchRows = 8;                    // rows per pass = warps per CTA
constexpr int kMarchThreads = 32 * kMarchRows;
constexpr int kMarchCols = 30;                   // destination columns per strip
constexpr int kMarchPostRows = kMarchRows + 2;   // ring of collided rows
constexpr int kMarchPhiRows = 2 * kMarchRows;    // ring of phi rows: two blocks of a pass each
constexpr int kMarchPW = 40;                     // phi ring row: columns xa .. xa + 39
constexpr int kMarchSN = kMarchPostRows * 32;
constexpr int kMarchPN = kMarchPhiRows * kMarchPW;

// Own-population loads of the march: plain loads after the phi barrier, or the same loads of
// boxes a TMA prefetch brought into L2 kMarchAhead passes ahead (when the step's buffers have
// tensor maps).
enum : int { MARCH_PLAIN = 0, MARCH_PREFETCH = 1 };
constexpr int kMarchAhead = 1;

// Shared memory of a march CTA: the collided ring, the phi ring (at a 128-byte boundary:
// TMA destination), the pre-collision h of warp kMarchRows - 1 for two passes, and the
// mbarrier of the phi ring's TMA loads.
template <bool FLOW>
__host__ __device__ constexpr size_t march_smem_bytes() {
  return sizeof(float) * (PostTile::floats<FLOW>(kMarchSN) + kMarchPN + 2 * 9 * 32) + 8;
}
static_assert(PostTile::floats<true>(kMarchSN) % 32 == 0 && PostTile::floats<false>(kMarchSN) % 32 == 0,
              "phi ring of the march not at a 128-byte boundary");
static_assert((kMarchRows * kMarchPW * 4) % 128 == 0, "phi ring block not 128-byte aligned");

__host__ __device__ constexpr int march_strips(int nx) { return (nx + kMarchCols - 1) / kMarchCols; }

// phi around a collided node in the phi ring: rows r0, r1, r2 (start indices of the ring rows
// below, at and above the node) and the node's column c.
struct RingView {
  const float* s;
  int r0, r1, r2, c;
  __device__ __forceinline__ float operator()(int dx, int dy) const {
    return s[(dy < 0 ? r0 : (dy > 0 ? r2 : r1)) + c + dx];
  }
  __device__ __forceinline__ bool ok() const {
    return in_range(r0 + c - 1, kMarchPN, OOB_SHARED) && in_range(r0 + c + 1, kMarchPN, OOB_SHARED) &&
           in_range(r1 + c - 1, kMarchPN, OOB_SHARED) && in_range(r1 + c + 1, kMarchPN, OOB_SHARED) &&
           in_range(r2 + c - 1, kMarchPN, OOB_SHARED) && in_range(r2 + c + 1, kMarchPN, OOB_SHARED);
  }
};

// Rows [r_begin, r_end) of the strip starting at grid column X0, by the whole CTA.
// Pass k (k = -1 is the prologue) collides rows r0 + 1 .. r0 + 8 (r0 = r_begin + 8k; warp w
// row r0 + 1 + w) and pulls rows r0 .. r0 + 7: warps 0..6 their own collided row, warp 7 the
// row it collided in the pass before (its pre-collision h kept in shared memory). The pull
// of row r reads the collided rows r - 1 .. r + 1, all in the ring of kMarchPostRows rows.
// phi^n comes in blocks of 8 rows: block k (rows r0 + 2 .. r0 + 9) is loaded while pass k - 1
// pulls, into half (k + 1) & 1 of a 16-row ring (grid row r at ring row (r - r_begin + 6) & 15,
// grid column xa + c at ring column c, xa = (X0 - 2) rounded down to a multiple of 4), so a
// pass's collisions find rows r0 .. r0 + 9 there. A CTA away from the grid faces whose step
// has tensor maps loads each block as one TMA box, issued by thread 0 and completing on an
// mbarrier; the others copy their rows with cp.async (ghost rows and columns resolved).
// PREF: thread 0 prefetches the populations of pass k + kMarchAhead into L2 as pass k starts.
template <bool FLOW, class S, int MODE, bool EDGE>
__device__ __forceinline__ void march_range(const Consts& C, const StepPtrs& P, int X0,
                                            int r_begin, int r_end, float* smem) {
  constexpr bool PREF = MODE == MARCH_PREFETCH;
  const PostTile post = PostTile::at<FLOW>(smem, kMarchSN);
  float* sphi = smem + PostTile::floats<FLOW>(kMarchSN);
  float* stash = sphi + kMarchPN;  // [2][9][32]
  uint64_t* bar = reinterpret_cast<uint64_t*>(stash + 2 * 9 * 32);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int X = X0 - 1 + lane;
  const int xa = (X0 - 2) & ~3;  // grid column of ring column 0 (16-byte aligned)
  const int po = X0 - 2 - xa;    // ring column of grid column X0 - 2
  const bool tphi = !EDGE && P.tm != nullptr;
  if (tphi) {
    if (threadIdx.x == 0) mbar_init(bar);
    __syncthreads();
  }
  if (PREF && threadIdx.x == 0)
    for (int j = 0; j < kMarchAhead && r_begin + kMarchRows * j < r_end; ++j)
      prefetch_issue<FLOW, S>(P, X0, r_begin + kMarchRows * j + 1);
  const bool xin = !EDGE || (X0 >= 2 && X0 + 32 <= C.nx);
  // collided ring: the row of warp w in pass k is ring row (pb + w) mod kMarchPostRows,
  // pb = (8k + 2) mod 10 (ring row 0: row r_begin - 1), kept incrementally
  const auto wrapP = [](int v) { return v < 0 ? v + kMarchPostRows : (v >= kMarchPostRows ? v - kMarchPostRows : v); };
  int pb = (2 - kMarchRows + 2 * kMarchPostRows) % kMarchPostRows;
  const auto phi_slot = [&](int r) { return (r - r_begin + 6) & (kMarchPhiRows - 1); };
  // phi^n block kk (rows r_begin + 8 kk + 2 .. + 9; the prologue kk = -1 needs only the last
  // four) into ring half (kk + 1) & 1
  const auto phi_block = [&](int kk) {
    float* half = sphi + ((kk + 1) & 1) * kMarchRows * kMarchPW;
    const int y0 = r_begin + kMarchRows * kk + 2;
    if (tphi) {
      if (threadIdx.x == 0) {
        mbar_expect(bar, kMarchRows * kMarchPW * sizeof(float));
        tma_load_2d(half, P.tm + 5, xa, y0, bar);
      }
      return;
    }
    const int rl = y0 + w;
    if ((kk >= 0 || w >= kMarchRows - 4) && rl <= r_end + 1 && (!EDGE || rl <= C.ny + 1)) {
      float* row = half + w * kMarchPW + po;
      const bool yin = !EDGE || (rl >= 0 && rl < C.ny);
      for (int c = lane; c < 34; c += 32) {
        if (!in_range(row - sphi + c, kMarchPN, OOB_SHARED)) continue;
        const int xg = X0 - 2 + c;
        if (xin && yin) {
          cp_async_plane(row + c, P.phi_n, rl * C.pitch + xg, (long long)C.pitch * C.ny);
        } else {
          int gx, gy;
          float v = -1.0f;
          if (xg > C.nx + 1) {
            v = 0.0f;  // beyond the grid's halo (ragged last strip): never read
          } else if (axis_phi(xg, C.nx, C.bc[0], C.bc[1], gx) &&
                     axis_phi(rl, C.ny, C.bc[2], C.bc[3], gy)) {
            v = ldg_plane(P.phi_n, (long long)gy * C.pitch + gx, (long long)C.pitch * C.ny);
          }
          row[c] = v;
        }
      }
    }
  };
  phi_block(-1);
  for (int k = -1;; ++k) {
    const int r0 = r_begin + kMarchRows * k;
    const int rc = r0 + 1 + w;  // collision row of this warp
    // (an interior CTA's rows and columns all lie inside the grid)
    const bool collide = (k >= 0 || w >= kMarchRows - 2) && rc <= r_end &&
                         (!EDGE || (rc <= C.ny && X <= C.nx));
    const int sc = wrapP(pb + w);  // collided-ring row of rc
    if (PREF && threadIdx.x == 0 && k >= 0 && r0 + kMarchRows * kMarchAhead < r_end)
      prefetch_issue<FLOW, S>(P, X0, r0 + kMarchRows * kMarchAhead + 1);

    // ---- A: phi block k, loaded during the pass before, is in the ring ----
    if (tphi)
      mbar_wait(bar, (k + 1) & 1);
    else
      cp_async_wait_all();
    __syncthreads();

    // ---- B: collide row rc ----
    float hown[9];
    if (collide) {
      const auto view_at = [&](int shx, int shy) {
        const int q = phi_slot(rc + shy);  // phi ring row of the mapped row
        return RingView{sphi, ((q - 1) & (kMarchPhiRows - 1)) * kMarchPW, q * kMarchPW,
                        ((q + 1) & (kMarchPhiRows - 1)) * kMarchPW, lane + 1 + shx + po};
      };
      collide_source<FLOW, S, true, 1, decltype(view_at), EDGE>(C, P, X, rc, sc * 32 + lane,
                                                                view_at, post, hown);
      if (w == kMarchRows - 1) {
        float* st = stash + (k & 1) * 9 * 32;
#pragma unroll
        for (int a = 0; a < 9; ++a) st[a * 32 + lane] = hown[a];
      }
    }
    __syncthreads();
    // Block k + 1 replaces the ring half of block k - 1 (rows r0 - 6 .. r0 + 1), which no
    // collision reads any more; the pull does not read the phi ring. The last pass loads
    // none, so no copy is in flight when the CTA ends.
    if (r0 + kMarchRows < r_end) phi_block(k + 1);
    // FP32 (latency-bound): this thread's node of the next pass is prefetched into L1 while
    // this pass pulls; the issue-bound 16-bit steps rely on the TMA prefetch into L2 alone
    if (!Storage<S>::DEV && !EDGE && rc + kMarchRows <= r_end) {
      const int rn = rc + kMarchRows;
      const int ndn = rn * (int)C.rstride + X;
#pragma unroll
      for (int p = 0; p < 4; ++p) prefetch_l1(static_cast<const float4*>(P.rin[p]) + ndn);
      prefetch_l1(static_cast<const float2*>(P.rin[4]) + ndn);
      if (FLOW) {
        prefetch_l1(static_cast<const float4*>(P.rin[5]) + ndn);
        prefetch_l1(static_cast<const float4*>(P.rin[6]) + ndn);
        prefetch_l1(static_cast<const float*>(P.rin[7]) + ndn);
      }
      prefetch_l1(P.phi_nm1 + (rn * C.pitch + X));
    }

    // ---- C: pull row rp ----
    if (k >= 0) {
      const int rp = w < kMarchRows - 1 ? rc : r0;
      if (rp < r_end && lane >= 1 && lane <= kMarchCols && (!EDGE || (rp < C.ny && X < C.nx))) {
        if (w == kMarchRows - 1) {
          const float* st = stash + ((k - 1) & 1) * 9 * 32;
#pragma unroll
          for (int a = 0; a < 9; ++a) hown[a] = st[a * 32 + lane];
        }
        // collided-ring row of rp: sc (warps 0..6), or that of r0 (warp 7)
        const int sp = w < kMarchRows - 1 ? sc : wrapP(pb - 1);
        const int s_m = wrapP(sp - 1) * 32 + lane;
        const int s_0 = sp * 32 + lane;
        const int s_p = wrapP(sp + 1) * 32 + lane;
        if (in_range(s_m - 1, kMarchSN, OOB_SHARED) && in_range(s_0 + 1, kMarchSN, OOB_SHARED) &&
            in_range(s_p + 1, kMarchSN, OOB_SHARED))
          pull_store<FLOW, S>(C, P, X, rp,
                              [&](int a) {
                                const int cy = cy_of(a);
                                return (cy > 0 ? s_m : (cy < 0 ? s_p : s_0)) - cx_of(a);
                              },
                              post, hown);
      }
    }
    pb = wrapP(pb + kMarchRows);
    if (r0 + kMarchRows >= r_end) break;  // rows r_begin .. r0 + 7 are done
  }
}

// Rows of the strip segment a march CTA walks (Consts::seg_rows, chosen on the host): tall
// enough that the two extra rows collided where a segment starts cost little, short enough
// that a launch has a few waves of CTAs. CTAs are numbered strip-fastest, so the CTAs
// resident at one time cover whole bands of rows, and neighbouring strips (which re-read
// each other's edge columns) run side by side.
constexpr int kMarchMaxSegRows = 64;

// One CTA per (strip, segment): blockIdx.x the strip, blockIdx.y the segment. Held to 64
// registers (4 CTAs of 256 threads per SM).
// A CTA whose phi columns X0 - 2 .. X0 + 31 and rows r0 - 2 .. r1 + 1 all lie inside the grid
// needs no ghost resolution: it runs the march compiled without it (EDGE = false).
__device__ __forceinline__ bool march_interior(const Consts& C, int X0, int r0, int r1) {
  return X0 >= 2 && X0 + 32 <= C.nx && r0 >= 2 && r1 + 2 <= C.ny;
}

template <bool FLOW, class S, int MODE>
__device__ __forceinline__ void march_cta(const Consts& C, const StepPtrs& P, int X0, int r0,
                                          int r1, float* smem) {
  if (march_interior(C, X0, r0, r1))
    march_range<FLOW, S, MODE, false>(C, P, X0, r0, r1, smem);
  else
    march_range<FLOW, S, MODE, true>(C, P, X0, r0, r1, smem);
}

template <bool FLOW, class S, int MODE>
__global__ void __launch_bounds__(kMarchThreads, 4) march_kernel(const Consts C, const StepPtrs P) {
  extern __shared__ __align__(128) float march_smem[];
  const int H = C.seg_rows, r0 = blockIdx.y * H;
  march_cta<FLOW, S, MODE>(C, P, blockIdx.x * kMarchCols, r0, min(C.ny, r0 + H), march_smem);
}

// ---- many grids in one launch ----------------------------------------------------------
// Shapes a member grid of a batched launch can use; the autotuner picks one per grid size.
// Shape 0 is the column march (one persistent wave over all its members); 1..3 are 2D tiles
// of 256 threads, each its own kernel instantiation launched with exactly its shared memory.
constexpr int kNumShapes = 4;
__host__ __device__ constexpr int shape_tx(int s) { return s == 1 ? 32 : s == 2 ? 64 : 16; }
__host__ __device__ constexpr int shape_ty(int s) { return s == 1 ? 8 : s == 2 ? 4 : 16; }

// One member grid of a batched launch: its constants, the buffer roles of this step and its
// tile count per row in the launch's shape (march: its strip count).
struct BatchDesc {
  Consts C;
  StepPtrs P;
  int tiles_x;
  int pad_;
};

// Parameter block of one batched launch: up to kBatchMaxMembers grids, list position k owning
// work units start[k] .. start[k+1]-1 (tiles, row-major within the grid; march: (strip, row)
// pairs, strip-major). It travels as a __grid_constant__ kernel parameter, so the descriptors
// sit in the constant bank (no device buffer to upload, nothing to race with launches still
// queued) and the block stays within the 32,764-byte parameter limit.
constexpr int kBatchMaxMembers = LBMICE_BATCH_MAX_PER_LAUNCH;
struct BatchLaunch {
  int n;
  long long tile_start[kBatchMaxMembers + 1];
  BatchDesc d[kBatchMaxMembers];
};
static_assert(sizeof(BatchLaunch) <= 32764, "kernel parameter limit");

// Last list position whose first unit is <= t.
__device__ __forceinline__ int batch_member_of(const BatchLaunch& L, long long t) {
  int lo = 0, hi = L.n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (L.tile_start[mid] <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// One CTA per tile of a batched launch: the owning grid, then the single-grid tile code. A
// tile beyond its grid (a malformed block) is skipped.
template <int TX, int TY, bool FLOW, class S>
__global__ void __launch_bounds__(TX* TY, 4) batch_step_kernel(const __grid_constant__ BatchLaunch L) {
  extern __shared__ __align__(16) float smem[];
  const long long t = blockIdx.x;
  const int m = batch_member_of(L, t);
  const BatchDesc& d = L.d[m];
  const int local = (int)(t - L.tile_start[m]);
  const int tyi = local / d.tiles_x, txi = local - tyi * d.tiles_x;
  if (local < 0 || tyi * TY >= d.C.ny) return;
  // no own-node preload here: the batched tile is more issue-bound than the single-grid one
  step_tile<TX, TY, FLOW, S, 1, false>(d.C, d.P, txi * TX, tyi * TY, smem);
}

// One CTA per (strip, segment) of the members of a march launch, numbered member by member,
// strip-fastest within a member; the members' populations are prefetched as in march_kernel.
template <bool FLOW, class S, int MODE>
__global__ void __launch_bounds__(kMarchThreads, 4) batch_march_kernel(const __grid_constant__ BatchLaunch L) {
  extern __shared__ __align__(128) float march_smem[];
  const long long t = blockIdx.x;
  const int m = batch_member_of(L, t);
  const BatchDesc& d = L.d[m];
  const int local = (int)(t - L.tile_start[m]);
  const int seg = local / d.tiles_x, strip = local - seg * d.tiles_x;
  const int H = d.C.seg_rows, r0 = seg * H;
  if (local < 0 || r0 >= d.C.ny) return;
  march_cta<FLOW, S, MODE>(d.C, d.P, strip * kMarchCols, r0, min(d.C.ny, r0 + H), march_smem);
}

}  // namespace lbmice
