// The fused collide-stream kernel: one launch advances h, g and f by one time step
// (arXiv 2101.07163, Sec. 2.2.1-2.2.3) over the whole grid.
//
// Each CTA owns a TX x TY tile of destination nodes and works in three phases:
//   A. phi^n of the tile plus a two-node halo (ghosts resolved) -> shared memory;
//   B. every source node of the tile plus a one-node halo is collided once: moments, the
//      E4 gradient from the shared phi tile, a_s and the anisotropic flux, the drag, and the
//      27 post-collision populations, which go to shared memory (h already divided by
//      a_s^2, together with 1 - 1/a_s^2, so the pull of Eq. (d) is one FMA). Interior nodes
//      keep their own pre-collision h in registers;
//   C. each destination pulls its 27 populations from the shared tile, applies Eq. (d),
//      writes h, g, f and phi^{n+1} = sum h to HBM.
// Global loads and stores of phases B and C are row-coalesced (consecutive threads own
// consecutive x). HBM traffic per node: 27 populations in and out, phi^n, phi^{n-1} in,
// phi^{n+1} out; halo re-reads hit L2.
#pragma once

#include <type_traits>

#include "../../include/lbmice.h"
#include "lbmice_device.cuh"

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
    return sizeof(float) * (size_t)(PN + (FLOW ? 27 : 18) * SN + SN);
  }
};

// Per-node coefficients of the three collisions, so that each direction costs a few FMAs:
//   phase field, Eq. (d)/(e): h* = h - (h - h^eq)/eta + w Q dt/tau0, h^eq = w (phi - 3 Dphi
//     c.N), stored divided by a_s^2:  h*/a_s^2 = a1 h + w (a2 - a3 c.N);
//   vapour: g* = g - (g - g^eq)/tau_g + w S dt, g^eq = w U (1 + 3 c.u*):
//     g* = b1 g + w (b2 + b3 c.u*);
//   flow: BGK to the second-order f^eq(rho, u*) plus Guo forcing of F = -k u*:
//     f* = c1 f + w (c2 + c.u* (c3 + c4 c.u*) + c.F (c5 + c6 c.u*)).
// Every product and sum is an explicit fmaf or round-to-nearest operation: the compiler may
// not contract them differently in different kernels, so every kernel that collides a node
// (single-grid or batched) produces the same bits.
template <bool FLOW>
struct FactoredCollision {
  float a1, a2, a3, b1, b2, b3, ux, uy;
  float c1 = 0.0f, c2 = 0.0f, c3 = 0.0f, c4 = 0.0f, c5 = 0.0f, c6 = 0.0f, Fx = 0.0f, Fy = 0.0f;
  __device__ __forceinline__ FactoredCollision(const Consts& C, float ph, float U, float rho,
                                               float inv_as2, float inv_eta, float srcQ,
                                               float inv_tg, float srcU, float k, float usx,
                                               float usy)
      : ux(usx), uy(usy) {
    a1 = __fmul_rn(1.0f - inv_eta, inv_as2);
    a2 = __fmul_rn(fmaf(ph, inv_eta, srcQ), inv_as2);
    a3 = __fmul_rn(__fmul_rn(C.Dphi3, inv_eta), inv_as2);
    b1 = 1.0f - inv_tg;
    b2 = fmaf(U, inv_tg, srcU);
    b3 = __fmul_rn(__fmul_rn(3.0f, U), inv_tg);
    if (FLOW) {
      Fx = -__fmul_rn(k, usx);
      Fy = -__fmul_rn(k, usy);
      const float uF = fmaf(usx, Fx, __fmul_rn(usy, Fy));
      const float uu = fmaf(usx, usx, __fmul_rn(usy, usy));
      const float r = __fmul_rn(rho, C.inv_tau_f);
      c1 = 1.0f - C.inv_tau_f;
      c2 = fmaf(r, fmaf(-1.5f, uu, 1.0f), -__fmul_rn(__fmul_rn(3.0f, C.guo), uF));
      c3 = __fmul_rn(3.0f, r);
      c4 = __fmul_rn(4.5f, r);
      c5 = __fmul_rn(3.0f, C.guo);
      c6 = __fmul_rn(9.0f, C.guo);
    }
  }
  // Populations given as deviations d_a = p_a - w_a M from the moments (phi, U, rho): each
  // collision is affine in p_a with slope a1, b1 or c1, so adding slope x M to the constant
  // term gives the same collided populations from the deviations.
  __device__ __forceinline__ void shift(float Mh, float Mg, float Mf) {
    a2 = fmaf(a1, Mh, a2);
    b2 = fmaf(b1, Mg, b2);
    if (FLOW) c2 = fmaf(c1, Mf, c2);
  }
  __device__ __forceinline__ float h(int a, float hv, float Nx, float Ny) const {
    return fmaf(hv, a1, __fmul_rn(w_of(a), fmaf(-a3, cdot(a, Nx, Ny), a2)));
  }
  __device__ __forceinline__ float g(int a, float gv) const {
    return fmaf(gv, b1, __fmul_rn(w_of(a), fmaf(b3, cdot(a, ux, uy), b2)));
  }
  __device__ __forceinline__ float f(int a, float fv) const {
    const float cu = cdot(a, ux, uy);
    const float t = fmaf(fmaf(c4, cu, c3), cu, c2);
    return fmaf(fv, c1, __fmul_rn(w_of(a), fmaf(cdot(a, Fx, Fy), fmaf(c6, cu, c5), t)));
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
  float h[9], g[9], f[9], php;
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
  in.valid = X < C.nx && Y < C.ny;
  if (!in.valid) return;
  const long long idx = (long long)Y * C.pitch + X;
  const long long nd = (long long)Y * C.rstride + X;
  const typename ST::T* __restrict__ pops = static_cast<const typename ST::T*>(P.pin);
  const long long np = (long long)C.pitch * C.ny;
  if constexpr (!ST::DEV) {
    load_lattice_f32(pops + PLANE_H * C.pstride, C.pstride, nd, in.h);
    load_lattice_f32(pops + PLANE_G * C.pstride, C.pstride, nd, in.g);
    if (FLOW) load_lattice_f32(pops + PLANE_F * C.pstride, C.pstride, nd, in.f);
  } else {
    in.h = ldg_vec(reinterpret_cast<const uint4*>(pops), nd, C.pstride);
    in.g = ldg_vec(reinterpret_cast<const uint4*>(pops + 9 * C.pstride), nd, C.pstride);
    in.U = ldg_plane(P.U_n, idx, np);
    if (FLOW) {
      in.f = ldg_vec(reinterpret_cast<const uint4*>(pops + 18 * C.pstride), nd, C.pstride);
      in.rho = ldg_plane(P.rho_n, idx, np);
    }
  }
  in.php = ldg_plane(P.phi_nm1, idx, np);
}

// Collide the source node at tile position (sx, sy) in [0, TX+2) x [0, TY+2), global
// coordinates (X, Y) in [-1, nx] x [-1, ny], and store its post-collision populations.
// Ghost positions take the collision of the node their face rule maps them to (directions
// mirrored across a free-slip wall), or the fixed inlet state.
template <int TX, int TY, bool FLOW, class S, bool OWN, int R>
__device__ __forceinline__ void collide_source(const Consts& C, const StepPtrs& P, int X, int Y,
                                               int sx, int sy, const float* __restrict__ sphi,
                                               float* __restrict__ spost,
                                               float* __restrict__ sB, float* hown,
                                               const OwnIn<S, FLOW>* pre = nullptr) {
  using T = Tile<TX, TY, R>;
  const int node = sy * T::SW + sx;
  if (!in_range(node, T::SN, OOB_SHARED)) return;
  int mx = X, my = Y, lx = sx, ly = sy;
  bool mirx = false, miry = false;
  int inlet = -1;
  if (X < 0 || X >= C.nx) {
    const int face = X < 0 ? 0 : 1;
    const int bc = X < 0 ? C.bc[0] : C.bc[1];
    if (bc == BC_PERIODIC) {
      mx = X < 0 ? X + C.nx : X - C.nx;
    } else {
      mx = X < 0 ? 0 : C.nx - 1;
      lx += X < 0 ? 1 : -1;
      mirx = bc == BC_FREESLIP;
      if (bc == BC_INLET) inlet = face;
    }
  }
  if (Y < 0 || Y >= C.ny) {
    const int face = Y < 0 ? 2 : 3;
    const int bc = Y < 0 ? C.bc[2] : C.bc[3];
    if (bc == BC_PERIODIC) {
      my = Y < 0 ? Y + C.ny : Y - C.ny;
    } else {
      my = Y < 0 ? 0 : C.ny - 1;
      ly += Y < 0 ? 1 : -1;
      miry = bc == BC_FREESLIP;
      if (bc == BC_INLET && inlet < 0) inlet = face;
    }
  }
  using ST = Storage<S>;
  const long long idx = (long long)my * C.pitch + mx;
  const typename ST::T* __restrict__ pops = static_cast<const typename ST::T*>(P.pin);
  const long long nd = (long long)my * C.rstride + mx;

  if (inlet >= 0) {
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
        load_lattice_f32(pops + PLANE_F * C.pstride, C.pstride, nd, fv);
        rho = sum9(fv);
      }
    }
    const float uu = ux * ux + uy * uy;
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      const float cu = cdot(a, ux, uy);
      spost[(PLANE_H + a) * T::SN + node] = -w_of(a);
      spost[(PLANE_G + a) * T::SN + node] = w_of(a) * C.U_in * (1.0f + 3.0f * cu);
      if (FLOW)
        spost[(PLANE_F + a) * T::SN + node] =
            w_of(a) * rho * (1.0f + 3.0f * cu + 4.5f * cu * cu - 1.5f * uu);
    }
    sB[node] = 0.0f;
    return;
  }

  // ---- populations and moments at time n (Sec. 2.2) ----
  const int pc = (ly + R) * T::PW + (lx + R);
  if (!in_range(pc - R * (T::PW + 1), T::PN, OOB_SHARED) ||
      !in_range(pc + R * (T::PW + 1), T::PN, OOB_SHARED))
    return;
  const float ph = sphi[pc];
  // FP32: the populations. 16-bit: their deviations d_a = p_a - w_a M from the stored
  // moments M (phi, U, rho), with d_0 = -sum_{a>0} d_a; the moments are the stored ones and
  // the momentum is sum c_a d_a (the w_a M terms cancel exactly).
  float hv[9], gv[9], fv[9];
  float php, U, rho = 1.0f;
  if (OWN && pre && pre->valid) {  // loaded before the phi tile's barrier
    if constexpr (!ST::DEV) {
#pragma unroll
      for (int a = 0; a < 9; ++a) {
        hv[a] = pre->h[a];
        gv[a] = pre->g[a];
        if (FLOW) fv[a] = pre->f[a];
      }
    } else {
      deviations9<S>(pre->h, hv);
      deviations9<S>(pre->g, gv);
      U = pre->U;
      if (FLOW) {
        deviations9<S>(pre->f, fv);
        rho = pre->rho;
      }
    }
    php = pre->php;
  } else {
    if constexpr (!ST::DEV) {
      load_lattice_f32(pops + PLANE_H * C.pstride, C.pstride, nd, hv);
      load_lattice_f32(pops + PLANE_G * C.pstride, C.pstride, nd, gv);
      if (FLOW) load_lattice_f32(pops + PLANE_F * C.pstride, C.pstride, nd, fv);
    } else {
      const uint4* pv = reinterpret_cast<const uint4*>(pops);
      const long long np = (long long)C.pitch * C.ny;
      deviations9<S>(ldg_vec(pv, nd, C.pstride), hv);
      deviations9<S>(ldg_vec(pv + (9 * C.pstride) / 8, nd, C.pstride), gv);
      U = ldg_plane(P.U_n, idx, np);
      if (FLOW) {
        deviations9<S>(ldg_vec(pv + (18 * C.pstride) / 8, nd, C.pstride), fv);
        rho = ldg_plane(P.rho_n, idx, np);
      }
    }
    php = ldg_plane(P.phi_nm1, idx, (long long)C.pitch * C.ny);
  }
  if constexpr (!ST::DEV) {
    U = sum9(gv);
    if (FLOW) rho = sum9(fv);
  }
  float jx = 0.0f, jy = 0.0f;
  if (FLOW) {
    jx = sumcx9(fv);
    jy = sumcy9(fv);
  }

  // ---- gradient of phi (Sec. 3.1.1, Table 1) and anisotropy (Sec. 2.1) ----
  float gx, gy;
  if (R == 1) {  // E4 with six-fold anisotropy: the default, with no run-time variant branch
    const float pE = sphi[pc + 1], pW = sphi[pc - 1];
    const float pN = sphi[pc + T::PW], pS = sphi[pc - T::PW];
    const float pNE = sphi[pc + T::PW + 1], pNW = sphi[pc + T::PW - 1];
    const float pSE = sphi[pc - T::PW + 1], pSW = sphi[pc - T::PW - 1];
    gx = fmaf(kW1, pE - pW, __fmul_rn(kW2, (pNE - pNW) + (pSE - pSW)));
    gy = fmaf(kW1, pN - pS, __fmul_rn(kW2, (pNE - pSE) + (pNW - pSW)));
  } else {  // any stencil and fold, chosen at run time, on a phi tile of halo R + 1 = 3
    gradient_stencil<float>(C.stencil, [&](int dx, int dy) { return sphi[pc + dy * T::PW + dx]; },
                            gx, gy);
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
    for (int a = 0; a < 9; ++a) hown[a] = ST::DEV ? fmaf(w_of(a), ph, hv[a]) : hv[a];
  }
  if constexpr (!Storage<S>::DEV) {
    // FP32 storage: the factored collision (FactoredCollision), each collided population
    // stored as it is formed (no staging array: the kernel stays at 64 registers); the
    // free-slip mirror is a uniform branch, so the common path stores at fixed
    // shared-memory offsets
    FactoredCollision<FLOW> fc(C, ph, U, rho, inv_as2, inv_eta, srcQ, inv_tg, srcU, k, usx, usy);
    auto emit = [&](auto mirrored) {
      constexpr bool M = decltype(mirrored)::value;
#pragma unroll
      for (int a = 0; a < 9; ++a) {
        int am = a;
        if constexpr (M) {
          am = mirx ? mirx_of(a) : a;
          am = miry ? miry_of(am) : am;
        }
        spost[(PLANE_H + am) * T::SN + node] = fc.h(a, hv[a], Nx, Ny);
        spost[(PLANE_G + am) * T::SN + node] = fc.g(a, gv[a]);
        if (FLOW) spost[(PLANE_F + am) * T::SN + node] = fc.f(a, fv[a]);
      }
    };
    if (mirx || miry) emit(std::true_type{}); else emit(std::false_type{});
  } else {
    // 16-bit storage: the same factored collision applied to the deviations (its constant
    // terms shifted by the moments), staged in registers, then stored
    FactoredCollision<FLOW> fc(C, ph, U, rho, inv_as2, inv_eta, srcQ, inv_tg, srcU, k, usx, usy);
    fc.shift(ph, U, rho);
    float post[27];
  #pragma unroll
    for (int a = 0; a < 9; ++a) {
      post[PLANE_H + a] = fc.h(a, hv[a], Nx, Ny);
      post[PLANE_G + a] = fc.g(a, gv[a]);
      if (FLOW) post[PLANE_F + a] = fc.f(a, fv[a]);
    }
    constexpr int NQ = FLOW ? 27 : 18;
    if (!mirx && !miry) {
  #pragma unroll
      for (int q = 0; q < NQ; ++q) spost[q * T::SN + node] = post[q];
    } else {  // ghost behind a free-slip wall: directions mirrored
  #pragma unroll
      for (int q = 0; q < NQ; ++q) {
        int am = mirx ? mirx_of(q % 9) : q % 9;
        am = miry ? miry_of(am) : am;
        spost[(q - q % 9 + am) * T::SN + node] = post[q];
      }
    }
  }
  sB[node] = 1.0f - inv_as2;
}

// One TX x TY tile with origin (x0, y0), computed by the TX * TY threads of the CTA (thread
// tid owns node (x0 + tid % TX, y0 + tid / TX)). smem holds Tile<TX, TY, R>::smem_bytes.
// PRE: issue the own node's loads before the phi tile's barrier (OwnIn).
template <int TX, int TY, bool FLOW, class S, int R = 1, bool PRE = true>
__device__ __forceinline__ void step_tile(const Consts& C, const StepPtrs& P, int x0, int y0,
                                          float* smem) {
  using ST = Storage<S>;
  using T = Tile<TX, TY, R>;
  constexpr int H = T::H;
  float* sphi = smem;
  float* spost = sphi + T::PN;
  float* sB = spost + (FLOW ? 27 : 18) * T::SN;
  const int tid = threadIdx.x;
  const int tx = tid % TX, ty = tid / TX;

  // the own node's populations, in flight while the phi tile loads
  OwnIn<S, FLOW> own;
  if (PRE) own_load<S, FLOW>(C, P, x0 + tx, y0 + ty, own);
  else own.valid = false;

  // ---- A: phi^n with a halo of H = R + 1 nodes ----
  if (x0 >= H && y0 >= H && x0 + TX + H <= C.nx && y0 + TY + H <= C.ny) {
    // the halo lies inside the grid (almost every tile): no ghost resolution
    const float* __restrict__ pb = P.phi_n + (long long)(y0 - H) * C.pitch + (x0 - H);
    const int pitch = (int)C.pitch;
    for (int i = tid; i < T::PN; i += T::NT) {
      const int lx = i % T::PW, ly = i / T::PW;
      if (in_range((long long)(y0 - H + ly) * C.pitch + (x0 - H + lx),
                   (long long)C.pitch * C.ny, OOB_PLANE))
        sphi[i] = __ldg(pb + ly * pitch + lx);
    }
  } else
  for (int i = tid; i < T::PN; i += T::NT) {
    const int lx = i % T::PW, ly = i / T::PW;
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
  __syncthreads();

  // ---- B: collide the tile (own node per thread) and its one-node ring ----
  float hown[9];
  {
    const int X = x0 + tx, Y = y0 + ty;
    if (X <= C.nx && Y <= C.ny)
      collide_source<TX, TY, FLOW, S, true, R>(C, P, X, Y, tx + 1, ty + 1, sphi, spost, sB,
                                               hown, &own);
  }
  for (int r = tid; r < T::NRING; r += T::NT) {
    // ring order: bottom row, top row, then left and right columns
    int sx, sy;
    if (r < T::SW) { sx = r; sy = 0; }
    else if (r < 2 * T::SW) { sx = r - T::SW; sy = TY + 1; }
    else { const int k = r - 2 * T::SW; sy = 1 + (k >> 1); sx = (k & 1) ? TX + 1 : 0; }
    const int X = x0 - 1 + sx, Y = y0 - 1 + sy;
    if (X >= -1 && X <= C.nx && Y >= -1 && Y <= C.ny)
      collide_source<TX, TY, FLOW, S, false, R>(C, P, X, Y, sx, sy, sphi, spost, sB, nullptr);
  }
  __syncthreads();

  // ---- C: pull, Eq. (d) for h, write populations and phi^{n+1} ----
  const int X = x0 + tx, Y = y0 + ty;
  if (X >= C.nx || Y >= C.ny) return;  // (this thread has no node in this tile)
  const long long idx = (long long)Y * C.pitch + X;
  const long long np = (long long)C.pitch * C.ny;
  // the nine pull sources span tile positions ty..ty+2 x tx..tx+2
  if (!in_range(ty * T::SW + tx, T::SN, OOB_SHARED) ||
      !in_range((ty + 2) * T::SW + tx + 2, T::SN, OOB_SHARED))
    return;
  float hn[9];
  if constexpr (!ST::DEV) {
    // FP32 storage: each lattice's pulled populations go back as two float4 and a float
    float gn[9], fn[9];
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      const int src = (ty + 1 - cy_of(a)) * T::SW + (tx + 1 - cx_of(a));
      hn[a] = fmaf(hown[a], sB[src], spost[(PLANE_H + a) * T::SN + src]);
      gn[a] = spost[(PLANE_G + a) * T::SN + src];
      if (FLOW) fn[a] = spost[(PLANE_F + a) * T::SN + src];
    }
    float* __restrict__ po = static_cast<float*>(P.pout);
    const long long nd = (long long)Y * C.rstride + X;
    store_lattice_f32(po + PLANE_H * C.pstride, C.pstride, nd, hn);
    store_lattice_f32(po + PLANE_G * C.pstride, C.pstride, nd, gn);
    if (FLOW) store_lattice_f32(po + PLANE_F * C.pstride, C.pstride, nd, fn);
    st_plane(P.phi_np1, idx, np, sum9(hn));
  } else {
    // 16-bit storage: the moments of the pulled populations are stored in FP32 and the
    // moving populations as deviations from them
    float gn[9], fn[9];
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      const int src = (ty + 1 - cy_of(a)) * T::SW + (tx + 1 - cx_of(a));
      hn[a] = fmaf(hown[a], sB[src], spost[(PLANE_H + a) * T::SN + src]);
      gn[a] = spost[(PLANE_G + a) * T::SN + src];
      if (FLOW) fn[a] = spost[(PLANE_F + a) * T::SN + src];
    }
    const float phin = sum9(hn);
    st_plane(P.phi_np1, idx, np, phin);
    typename ST::T* __restrict__ pout = static_cast<typename ST::T*>(P.pout);
    const long long nd = (long long)Y * C.rstride + X;
    store9<S>(pout, 0, C.pstride, nd, phin, hn);
    const float Un = sum9(gn);
    st_plane(P.U_np1, idx, np, Un);
    store9<S>(pout, 1, C.pstride, nd, Un, gn);
    if (FLOW) {
      const float rn = sum9(fn);
      st_plane(P.rho_np1, idx, np, rn);
      store9<S>(pout, 2, C.pstride, nd, rn, fn);
    }
  }
}

// One CTA per TX x TY tile. FP32 storage is held to 64 registers (4 CTAs of 256 threads per
// SM, the measured optimum); the 16-bit forms keep the compiler's own allocation, which a
// minimum-blocks bound would change.
template <int TX, int TY, bool FLOW, class S, int R>
__global__ std::enable_if_t<!Storage<S>::DEV> __launch_bounds__(TX* TY, 4)
    step_kernel(const Consts C, const StepPtrs P) {
  extern __shared__ float smem[];
  step_tile<TX, TY, FLOW, S, R>(C, P, blockIdx.x * TX, blockIdx.y * TY, smem);
}
template <int TX, int TY, bool FLOW, class S, int R>
__global__ std::enable_if_t<Storage<S>::DEV> __launch_bounds__(TX* TY)
    step_kernel(const Consts C, const StepPtrs P) {
  extern __shared__ float smem[];
  step_tile<TX, TY, FLOW, S, R>(C, P, blockIdx.x * TX, blockIdx.y * TY, smem);
}

// ---- many grids in one launch ----------------------------------------------------------
// Tile shapes of 256 threads that the batched kernel can use for a member grid; the
// autotuner picks one per grid size. Each shape is its own kernel instantiation, launched
// with exactly its shared memory (a larger request shrinks the L1 left for the pull).
constexpr int kNumShapes = 3;
__host__ __device__ constexpr int shape_tx(int s) { return s == 0 ? 32 : s == 1 ? 64 : 16; }
__host__ __device__ constexpr int shape_ty(int s) { return s == 0 ? 8 : s == 1 ? 4 : 16; }

// One member grid of a batched launch: its constants, the buffer roles of this step and its
// tile count per row in the launch's shape.
struct BatchDesc {
  Consts C;
  StepPtrs P;
  int tiles_x;
  int pad_;
};

// Parameter block of one batched launch: up to kBatchMaxMembers grids, list position k owning
// tiles tile_start[k] .. tile_start[k+1]-1 (row-major within the grid). It travels as a
// __grid_constant__ kernel parameter, so the descriptors sit in the constant bank (no device
// buffer to upload, nothing to race with launches still queued) and the block stays within
// the 32,764-byte parameter limit.
constexpr int kBatchMaxMembers = LBMICE_BATCH_MAX_PER_LAUNCH;
struct BatchLaunch {
  int n;
  int tile_start[kBatchMaxMembers + 1];
  BatchDesc d[kBatchMaxMembers];
};
static_assert(sizeof(BatchLaunch) <= 32764, "kernel parameter limit");

// One CTA per tile of a batched launch: binary search for the owning grid, then the
// single-grid tile code. A tile beyond its grid (a malformed block) is skipped.
template <int TX, int TY, bool FLOW, class S>
__global__ void __launch_bounds__(TX* TY, 4) batch_step_kernel(const __grid_constant__ BatchLaunch L) {
  extern __shared__ float smem[];
  const int t = blockIdx.x;
  int lo = 0, hi = L.n - 1;  // last list position whose first tile is <= t
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (L.tile_start[mid] <= t) lo = mid; else hi = mid - 1;
  }
  const BatchDesc& d = L.d[lo];
  const int local = t - L.tile_start[lo];
  const int tyi = local / d.tiles_x, txi = local - tyi * d.tiles_x;
  if (local < 0 || tyi * TY >= d.C.ny) return;
  // no own-node preload here: the batched tile is more issue-bound than the single-grid one
  // and measured 2.7% faster without it
  step_tile<TX, TY, FLOW, S, 1, false>(d.C, d.P, txi * TX, tyi * TY, smem);
}

}  // namespace lbmice
