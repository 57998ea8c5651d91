// Discrete adjoint (reverse mode) of the fused FP32 step of the coupled lattice-Boltzmann
// ice-crystal model (arXiv 2101.07163, Sec. 2.2), on periodic grids.
//
// The forward step maps the state S^n = (populations p^n, phi^n plane, phi^{n-1} plane) to
//   p^{n+1} = pull(collide(p^n, phi^n, phi^{n-1})),  phi^{n+1} = sum_a h_a^{n+1},  and the
//   history plane of S^{n+1} is phi^n.
// Every coupling reads phi from the phi^n plane (the node's phi and the E4 gradient), which
// equals sum_a h_a^n on every trajectory, so derivatives along trajectories are the same
// whichever of the two is differentiated. Given the adjoint of S^{n+1} (pb, Phib, Psib), one
// reverse step produces the adjoint of S^n in two or three kernels:
//   adj_collide_kernel (per node x): gathers the adjoints of the pulled values from the
//     downstream nodes x + c_a, recomputes the collision of x and runs it backwards: writes the
//     population adjoints, the node-local part of the phi^n adjoint, the adjoint of the
//     node's E4 gradient and the adjoint of phi^{n-1}; accumulates the parameter adjoints
//     (FP32 within a warp, FP64 across warps, blocks and steps; one slot per block:
//     deterministic). The pull's own-population term h_a^{n+1}(y) = h_a^n(y) B(y - c_a) + ...
//     (B = 1 - 1/a_s^2) is added in one of two ways:
//   - grids whose reverse working set fits in L2: adj_collide writes B, then adj_pull_kernel
//     (per node y) adds the term to the h adjoints (read-modify-write, L2-resident) and
//     gathers the transpose of the E4 stencil;
//   - larger grids (FUSED): adj_b_kernel writes B first, adj_collide adds the term as it
//     writes the h adjoints (each written once), and adj_stencil_kernel gathers the
//     transpose of the E4 stencil.
//   Both give the same bits.
//   adj_stencil_kernel (per node y): the phi^n adjoint, node-local part plus the transpose of
//     the E4 stencil gathered from the gradient adjoints of the neighbours.
// Non-differentiable points are taken as the branch the forward step takes: below the
// |grad phi|^2 threshold a_s = 1 and N = 0 do not depend on the gradient or on eps; q(phi)
// has zero slope where the clamp to [0, 2] is active.
#pragma once

#include "lbmice_device.cuh"

namespace lbmice {

// Buffers of one reverse step. The forward populations are in the step's node-interleaved
// FP32 layout (load_hg_f32, load_lattice_f32, f32_pop_index); their adjoints are plain planes,
// q * pstride + y * rstride + x; every other plane is [ny][pitch].
struct AdjPtrs {
  const float* pops;     // forward state n: populations
  const float* phi_n;    // forward state n: the phi^n plane
  const float* phi_nm1;  // forward state n: the phi^{n-1} plane
  const float* pb_in;    // adjoint of p^{n+1}
  const float* Phib_in;  // adjoint of the phi^{n+1} plane
  const float* Psib_in;  // adjoint of the history plane of S^{n+1} (which holds phi^n)
  float* pb_out;         // adjoint of p^n
  float* Phib_out;       // adjoint of the phi^n plane
  float* Psib_out;       // adjoint of the phi^{n-1} plane
  float* phib_loc;       // scratch: node-local phi^n adjoint plus Psib_in
  float* gbx;            // scratch: adjoint of the node's E4 gradient, x component
  float* gby;            //   and y component
  float* Bn;             // scratch: B = 1 - 1/a_s^2 of every node (adj_b_kernel, or the
                         // separate form's adj_collide_kernel)
  double* partial;       // [blocks][kAdjParams] parameter adjoints, accumulated over steps
};

// Parameter adjoints accumulated per block: the kernel constants eps, kappa_N 6 eps,
// 3 D dt/dx^2 and lambda.
constexpr int kAdjParams = 4;
enum : int { ADJ_EPS = 0, ADJ_KN6EPS = 1, ADJ_DLAT3 = 2, ADJ_LAMBDA = 3 };

__device__ __forceinline__ int wrap_p(int v, int n) { return v >= n ? v - n : v; }
__device__ __forceinline__ int wrap_m(int v, int n) { return v < 0 ? v + n : v; }
__device__ __forceinline__ int step_to(int v, int c, int n) {
  return c > 0 ? wrap_p(v + 1, n) : (c < 0 ? wrap_m(v - 1, n) : v);
}

// Sum of v over the block into out[k] (threads 0..kAdjParams-1 add). Each thread holds one
// node's FP32 terms: a warp sums its 32 in FP32 (a five-level tree, error below 3e-7 of the
// sum of magnitudes), and only the warp sums and the running total are FP64 -- the FP64
// pipe of this part retires about one warp instruction per 64 cycles per scheduler, so an
// FP64 tree per thread would dominate the kernel.
__device__ __forceinline__ void block_accumulate(const float* v, double* out) {
  __shared__ double red[8][kAdjParams];
#pragma unroll
  for (int k = 0; k < kAdjParams; ++k) {
    float s = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][k] = (double)s;
  }
  __syncthreads();
  if (threadIdx.x < kAdjParams) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w][threadIdx.x];
    out[threadIdx.x] += s;
  }
}

// B = 1 - 1/a_s^2 at node (x, y) of a periodic grid, from the E4 gradient of phi^n, with
// the arithmetic of the collision adjoint's recomputation below.
__device__ __forceinline__ float adj_node_B(const Consts& C, const float* __restrict__ phi,
                                            int x, int y) {
  const int PI = C.pitch;  // every plane index is below 2^31 (lbmice_create)
  const int xp = wrap_p(x + 1, C.nx), xm = wrap_m(x - 1, C.nx);
  const int yp = wrap_p(y + 1, C.ny), ym = wrap_m(y - 1, C.ny);
  auto P = [&](int xx, int yy) { return __ldg(phi + (yy * PI + xx)); };
  const float pE = P(xp, y), pW = P(xm, y), pN = P(x, yp), pS = P(x, ym);
  const float pNE = P(xp, yp), pNW = P(xm, yp), pSE = P(xp, ym), pSW = P(xm, ym);
  const float gx = kW1 * (pE - pW) + kW2 * ((pNE - pNW) + (pSE - pSW));
  const float gy = kW1 * (pN - pS) + kW2 * ((pNE - pSE) + (pNW - pSW));
  const float s2 = gx * gx + gy * gy;
  float as = 1.0f;
  if (s2 > 1e-12f) {
    const float rinv = rsqrtf(s2);
    const float nx = gx * rinv, ny = gy * rinv;
    const float X2 = nx * nx, Y2 = ny * ny;
    const float cos6 = X2 * X2 * X2 - 15.0f * X2 * X2 * Y2 + 15.0f * X2 * Y2 * Y2 - Y2 * Y2 * Y2;
    as = 1.0f + C.eps * cos6;
  }
  return 1.0f - __fdividef(1.0f, as * as);
}

// B of every node into the Bn plane, before the collision adjoint reads it at x - c_a.
__global__ void __launch_bounds__(256) adj_b_kernel(const Consts C, const AdjPtrs A) {
  const int x = blockIdx.x * 32 + (threadIdx.x & 31);
  const int y = blockIdx.y * 8 + (threadIdx.x >> 5);
  if (x >= C.nx || y >= C.ny) return;
  A.Bn[y * C.pitch + x] = adj_node_B(C, A.phi_n, x, y);
}

// Adjoint of the collision of every node (block 32 x 8, one thread per node). Held to 80
// registers for 3 CTAs per SM: the bytes of spills this costs the flow form are cheaper
// than the third CTA's latency hiding is worth (measured 128.6 -> 120.2 ms per reverse sweep).
// FUSED: adds the pull's own-population term to the h adjoints (B from adj_b_kernel); else
// writes B for adj_pull_kernel.
template <bool FLOW, bool FUSED>
__global__ void __launch_bounds__(256, 3) adj_collide_kernel(const Consts C, const AdjPtrs A) {
  const int x = blockIdx.x * 32 + (threadIdx.x & 31);
  const int y = blockIdx.y * 8 + (threadIdx.x >> 5);
  float part[kAdjParams] = {0.0f, 0.0f, 0.0f, 0.0f};
  if (x < C.nx && y < C.ny) {
    const float* __restrict__ pb_in = A.pb_in;  // the adjoint ping-pong buffers never alias
    float* __restrict__ pb_out = A.pb_out;
    // plane strides in 64 bits; node and plane indices below 2^31 (lbmice_create)
    const long long Q = C.pstride;
    const int R = (int)C.rstride, PI = C.pitch;
    const int xp = wrap_p(x + 1, C.nx), xm = wrap_m(x - 1, C.nx);
    const int yp = wrap_p(y + 1, C.ny), ym = wrap_m(y - 1, C.ny);
    const int ip = y * R + x;   // population offset of the node
    const int iq = y * PI + x;  // plane offset of the node

    // ---- forward recomputation of the node's collision (the step kernel's quantities, in
    //      their unfactored form; values agree with the kernel's to rounding) ----
    float hv[9], gv[9], fv[9];
    {
      float2 hg[9];
      load_hg_f32(A.pops, Q, ip, hg);
#pragma unroll
      for (int a = 0; a < 9; ++a) {
        hv[a] = hg[a].x;
        gv[a] = hg[a].y;
      }
    }
    if (FLOW) {
      load_lattice_f32(A.pops + 18 * Q, Q, ip, fv);
    } else {
#pragma unroll
      for (int a = 0; a < 9; ++a) fv[a] = 0.0f;
    }
    const float ph = __ldg(A.phi_n + iq);
    const float U = sum9(gv);
    float rho = 1.0f, jx = 0.0f, jy = 0.0f;
    if (FLOW) {
      rho = sum9(fv);
      jx = sumcx9(fv);
      jy = sumcy9(fv);
    }
    auto P = [&](int xx, int yy) { return __ldg(A.phi_n + (yy * PI + xx)); };
    const float pE = P(xp, y), pW = P(xm, y), pN = P(x, yp), pS = P(x, ym);
    const float pNE = P(xp, yp), pNW = P(xm, yp), pSE = P(xp, ym), pSW = P(xm, ym);
    const float gx = kW1 * (pE - pW) + kW2 * ((pNE - pNW) + (pSE - pSW));
    const float gy = kW1 * (pN - pS) + kW2 * ((pNE - pSE) + (pNW - pSW));
    const float s2 = gx * gx + gy * gy;
    const bool aniso_on = s2 > 1e-12f;
    float as = 1.0f, Nx = 0.0f, Ny = 0.0f, rinv = 0.0f, nx = 0.0f, ny = 0.0f;
    float X2 = 0.0f, Y2 = 0.0f, cos6 = 0.0f, sin6 = 0.0f, t = 0.0f;
    if (aniso_on) {
      rinv = rsqrtf(s2);
      nx = gx * rinv;
      ny = gy * rinv;
      X2 = nx * nx;
      Y2 = ny * ny;
      cos6 = X2 * X2 * X2 - 15.0f * X2 * X2 * Y2 + 15.0f * X2 * Y2 * Y2 - Y2 * Y2 * Y2;
      sin6 = nx * ny * (6.0f * X2 * X2 - 20.0f * X2 * Y2 + 6.0f * Y2 * Y2);
      as = 1.0f + C.eps * cos6;
      t = C.kNkeps * as * sin6;
      Nx = t * gy;
      Ny = -(t * gx);
    }
    const float as2 = as * as;
    const float inv_as2 = __fdividef(1.0f, as2);
    const float inv_eta = __fdividef(1.0f, C.Dphi3 * as2 + 0.5f);
    const float omp2 = 1.0f - ph * ph;
    const float srcQ = (ph - ph * ph * ph + C.lambda * U * omp2 * omp2) * C.dt_tau0;
    float usx = 0.0f, usy = 0.0f, k = 0.0f, inv = 0.0f, sfac = 0.0f;
    const float onep = 1.0f + ph;
    if (FLOW) {
      k = C.kdrag * rho * onep * onep * (1.0f - ph);
      inv = __fdividef(1.0f, rho + 0.5f * k);
      sfac = 0.5f * (1.0f - ph);
      usx = sfac * (jx * inv);
      usy = sfac * (jy * inv);
    }
    const float qraw = 1.0f - ph;
    const float q = fminf(fmaxf(qraw, 0.0f), 2.0f);
    const float inv_tg = __fdividef(1.0f, C.Dlat3 * q + 0.5f);
    const float Fx = -k * usx, Fy = -k * usy;
    const float uu = usx * usx + usy * usy;

    // ---- adjoints of the pulled values, gathered from the downstream nodes x + c_a ----
    // h: A_a = h*_a / a_s^2 reaches h_a^{n+1}(x + c_a), whose adjoint includes the phi^{n+1}
    // plane (phi^{n+1} = sum h^{n+1}); B = 1 - 1/a_s^2 multiplies h_a^n(x + c_a).
    float Ab[9], Gb[9], Fb[9];
    float Bb = 0.0f;
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      const int xs = step_to(x, cx_of(a), C.nx), ys = step_to(y, cy_of(a), C.ny);
      const int jp = ys * R + xs;
      const float hhat = __ldg(pb_in + (PLANE_H + a) * Q + jp) +
                         __ldg(A.Phib_in + (ys * PI + xs));
      Ab[a] = hhat;
      Bb += hhat * __ldg(A.pops + f32_pop_index(Q, jp, 0, a));
      Gb[a] = __ldg(pb_in + (PLANE_G + a) * Q + jp);
      Fb[a] = FLOW ? __ldg(pb_in + (PLANE_F + a) * Q + jp) : 0.0f;
    }

    // ---- phase field: A_a = h*_a inv_as2, B = 1 - inv_as2,
    //      h*_a = h_a - (h_a - heq_a) inv_eta + w_a srcQ, heq_a = w_a (phi - Dphi3 c_a.N) ----
    float phb = 0.0f, Ub = 0.0f;
    float inv_as2_b = -Bb, inv_eta_b = 0.0f, srcQ_b = 0.0f, Nxb = 0.0f, Nyb = 0.0f;
    float hb[9];
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      const float w = w_of(a);
      const float heq = w * (ph - C.Dphi3 * cdot(a, Nx, Ny));
      const float hs = hv[a] - (hv[a] - heq) * inv_eta + w * srcQ;
      inv_as2_b += Ab[a] * hs;
      const float hsb = Ab[a] * inv_as2;
      hb[a] = hsb * (1.0f - inv_eta);
      inv_eta_b -= hsb * (hv[a] - heq);
      const float heqb = hsb * inv_eta;
      srcQ_b += w * hsb;
      phb += w * heqb;
      Nxb -= C.Dphi3 * w * heqb * (float)cx_of(a);
      Nyb -= C.Dphi3 * w * heqb * (float)cy_of(a);
    }
    // inv_eta = 1/(Dphi3 as2 + 1/2), inv_as2 = 1/as2
    const float as2_b = -inv_eta_b * C.Dphi3 * inv_eta * inv_eta - inv_as2_b * inv_as2 * inv_as2;
    float as_b = 2.0f * as * as2_b;
    // srcQ = (phi - phi^3 + lambda U (1 - phi^2)^2) dt/tau0
    phb += srcQ_b * C.dt_tau0 * (1.0f - 3.0f * ph * ph - 4.0f * C.lambda * U * omp2 * ph);
    Ub += srcQ_b * C.dt_tau0 * C.lambda * omp2 * omp2;
    part[ADJ_LAMBDA] += srcQ_b * C.dt_tau0 * U * omp2 * omp2;
    // anisotropy: N = t (g_y, -g_x), t = kNkeps a_s sin6, a_s = 1 + eps cos6, n = g / |g|
    float gxb = 0.0f, gyb = 0.0f;
    if (aniso_on) {
      const float tb = Nxb * gy - Nyb * gx;
      gyb += Nxb * t;
      gxb -= Nyb * t;
      as_b += tb * C.kNkeps * sin6;
      const float sin6_b = tb * C.kNkeps * as;
      part[ADJ_KN6EPS] += tb * as * sin6;
      const float cos6_b = as_b * C.eps;
      part[ADJ_EPS] += as_b * cos6;
      const float Pp = 6.0f * X2 * X2 - 20.0f * X2 * Y2 + 6.0f * Y2 * Y2;
      const float X2b = cos6_b * (3.0f * X2 * X2 - 30.0f * X2 * Y2 + 15.0f * Y2 * Y2) +
                        sin6_b * nx * ny * (12.0f * X2 - 20.0f * Y2);
      const float Y2b = cos6_b * (-15.0f * X2 * X2 + 30.0f * X2 * Y2 - 3.0f * Y2 * Y2) +
                        sin6_b * nx * ny * (-20.0f * X2 + 12.0f * Y2);
      const float nxb = sin6_b * ny * Pp + 2.0f * nx * X2b;
      const float nyb = sin6_b * nx * Pp + 2.0f * ny * Y2b;
      const float dn = nxb * nx + nyb * ny;
      gxb += rinv * (nxb - dn * nx);
      gyb += rinv * (nyb - dn * ny);
    }

    // ---- vapour: g*_a = g_a - (g_a - geq_a) inv_tg + w_a srcU, geq_a = w_a U (1 + 3 c_a.u*) ----
    float inv_tg_b = 0.0f, srcU_b = 0.0f, usxb = 0.0f, usyb = 0.0f;
    float gb[9];
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      const float w = w_of(a);
      const float cu = cdot(a, usx, usy);
      const float geq = w * U * (1.0f + 3.0f * cu);
      gb[a] = Gb[a] * (1.0f - inv_tg);
      inv_tg_b -= Gb[a] * (gv[a] - geq);
      const float geqb = Gb[a] * inv_tg;
      srcU_b += w * Gb[a];
      Ub += geqb * w * (1.0f + 3.0f * cu);
      const float cub = geqb * w * U * 3.0f;
      usxb += cub * (float)cx_of(a);
      usyb += cub * (float)cy_of(a);
    }
    // srcU = -(L_sat/2)(phi - phi^{n-1})
    phb -= C.half_Lsat * srcU_b;
    const float phpb = C.half_Lsat * srcU_b;
    // inv_tg = 1/(Dlat3 q + 1/2); q = clamp(1 - phi, 0, 2)
    const float qb = -inv_tg_b * C.Dlat3 * inv_tg * inv_tg;
    part[ADJ_DLAT3] += -inv_tg_b * q * inv_tg * inv_tg;
    if (qraw >= 0.0f && qraw <= 2.0f) phb -= qb;

    // ---- flow: f*_a = f_a - (f_a - feq_a)/tau_f + force_a ----
    float fb[9];
    if (FLOW) {
      float rhob = 0.0f, uub = 0.0f, uFb = 0.0f, Fxb = 0.0f, Fyb = 0.0f;
#pragma unroll
      for (int a = 0; a < 9; ++a) {
        const float w = w_of(a);
        const float cu = cdot(a, usx, usy);
        const float cF = cdot(a, Fx, Fy);
        fb[a] = Fb[a] * (1.0f - C.inv_tau_f);
        const float feqb = Fb[a] * C.inv_tau_f;
        // feq_a = w rho (1 + 3 cu + 4.5 cu^2 - 1.5 uu)
        rhob += feqb * w * (1.0f + 3.0f * cu + 4.5f * cu * cu - 1.5f * uu);
        float cub = feqb * w * rho * (3.0f + 9.0f * cu);
        uub -= 1.5f * feqb * w * rho;
        // force_a = guo w (3 (cF - uF) + 9 cu cF)
        const float cFb = Fb[a] * C.guo * w * (3.0f + 9.0f * cu);
        cub += Fb[a] * C.guo * w * 9.0f * cF;
        uFb -= 3.0f * Fb[a] * C.guo * w;
        usxb += cub * (float)cx_of(a);
        usyb += cub * (float)cy_of(a);
        Fxb += cFb * (float)cx_of(a);
        Fyb += cFb * (float)cy_of(a);
      }
      // uu = us.us, uF = us.F, F = -k us
      usxb += 2.0f * usx * uub + Fx * uFb;
      usyb += 2.0f * usy * uub + Fy * uFb;
      Fxb += usx * uFb;
      Fyb += usy * uFb;
      const float kb0 = -(usx * Fxb + usy * Fyb);
      usxb -= k * Fxb;
      usyb -= k * Fyb;
      // us = sfac j inv
      const float sfacb = usxb * jx * inv + usyb * jy * inv;
      const float jxb = usxb * sfac * inv, jyb = usyb * sfac * inv;
      const float invb = usxb * sfac * jx + usyb * sfac * jy;
      phb -= 0.5f * sfacb;
      // inv = 1/(rho + k/2)
      const float denb = -invb * inv * inv;
      rhob += denb;
      const float kb = kb0 + 0.5f * denb;
      // k = kdrag rho (1+phi)^2 (1-phi)
      rhob += kb * C.kdrag * onep * onep * (1.0f - ph);
      phb += kb * C.kdrag * rho * onep * (1.0f - 3.0f * ph);
      // rho = sum f, j = sum c f
#pragma unroll
      for (int a = 0; a < 9; ++a)
        fb[a] += rhob + (float)cx_of(a) * jxb + (float)cy_of(a) * jyb;
    }
    // ---- outputs (U = sum g); FUSED: h adds the pull's own-population term ----
    const float Phb_own = FUSED ? __ldg(A.Phib_in + iq) : 0.0f;
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      if (FUSED) {
        const float hhat = __ldg(pb_in + (PLANE_H + a) * Q + ip) + Phb_own;
        const int xs = step_to(x, -cx_of(a), C.nx), ys = step_to(y, -cy_of(a), C.ny);
        pb_out[(PLANE_H + a) * Q + ip] = hb[a] + hhat * __ldg(A.Bn + (ys * PI + xs));
      } else {
        pb_out[(PLANE_H + a) * Q + ip] = hb[a];
      }
      pb_out[(PLANE_G + a) * Q + ip] = gb[a] + Ub;
      if (FLOW) pb_out[(PLANE_F + a) * Q + ip] = fb[a];
    }
    A.phib_loc[iq] = phb + __ldg(A.Psib_in + iq);
    A.gbx[iq] = gxb;
    A.gby[iq] = gyb;
    A.Psib_out[iq] = phpb;
    if (!FUSED) A.Bn[iq] = 1.0f - inv_as2;
  }
  const int slot = blockIdx.y * gridDim.x + blockIdx.x;
  block_accumulate(part, A.partial + (long long)slot * kAdjParams);
}

// Transpose of the E4 stencil at node (x, y): sum_e w_e (c_e . gb(y - e)), where the gradient
// at z reads phi(z + e) with weight w_e c_e (e = (1,0) is read by z = (x-1, y), and so on).
__device__ __forceinline__ float e4_transpose(const Consts& C, const float* __restrict__ gbx,
                                              const float* __restrict__ gby, int x, int y) {
  const int PI = C.pitch;
  const int xp = wrap_p(x + 1, C.nx), xm = wrap_m(x - 1, C.nx);
  const int yp = wrap_p(y + 1, C.ny), ym = wrap_m(y - 1, C.ny);
  auto GX = [&](int xx, int yy) { return __ldg(gbx + (yy * PI + xx)); };
  auto GY = [&](int xx, int yy) { return __ldg(gby + (yy * PI + xx)); };
  const float axis = kW1 * ((GX(xm, y) - GX(xp, y)) + (GY(x, ym) - GY(x, yp)));
  const float diag = kW2 * ((GX(xm, ym) - GX(xp, yp)) + (GX(xm, yp) - GX(xp, ym)) +
                            (GY(xm, ym) - GY(xp, yp)) + (GY(xp, ym) - GY(xm, yp)));
  return axis + diag;
}

// Own-population term of the pull and transpose of the E4 stencil (one thread per node y):
//   pb_out_h,a(y) += hhat_a(y) B(y - c_a),   hhat_a(y) = pb_in_h,a(y) + Phib_in(y);
//   Phib_out(y) = phib_loc(y) + sum_e w_e (c_e . gb(y - e)).
__global__ void __launch_bounds__(256) adj_pull_kernel(const Consts C, const AdjPtrs A) {
  const int x = blockIdx.x * 32 + (threadIdx.x & 31);
  const int y = blockIdx.y * 8 + (threadIdx.x >> 5);
  if (x >= C.nx || y >= C.ny) return;
  const long long Q = C.pstride;
  const int R = (int)C.rstride, PI = C.pitch;
  const int ip = y * R + x, iq = y * PI + x;
  const float Phb = __ldg(A.Phib_in + iq);
#pragma unroll
  for (int a = 0; a < 9; ++a) {
    const int xs = step_to(x, -cx_of(a), C.nx), ys = step_to(y, -cy_of(a), C.ny);
    const float hhat = __ldg(A.pb_in + (PLANE_H + a) * Q + ip) + Phb;
    A.pb_out[(PLANE_H + a) * Q + ip] += hhat * __ldg(A.Bn + (ys * PI + xs));
  }
  A.Phib_out[iq] = __ldg(A.phib_loc + iq) + e4_transpose(C, A.gbx, A.gby, x, y);
}

// The phi^n adjoint (one thread per node y), once every node's gradient adjoint is known:
//   Phib_out(y) = phib_loc(y) + sum_e w_e (c_e . gb(y - e)).
__global__ void __launch_bounds__(256) adj_stencil_kernel(const Consts C, const AdjPtrs A) {
  const int x = blockIdx.x * 32 + (threadIdx.x & 31);
  const int y = blockIdx.y * 8 + (threadIdx.x >> 5);
  if (x >= C.nx || y >= C.ny) return;
  const int iq = y * C.pitch + x;
  A.Phib_out[iq] = __ldg(A.phib_loc + iq) + e4_transpose(C, A.gbx, A.gby, x, y);
}

// Adjoint of the initialisation (equilibria of the moments phi0, U0, rho0, u0; Sec. 2.2 and
// the equilibrium initial state): h_a = w_a (phi0 - Dphi3 c_a.N(grad phi0)),
// g_a = w_a U0 (1 + 3 c_a.u0), f_a = w_a rho0 (1 + 3 c.u0 + 4.5 (c.u0)^2 - 1.5 u0.u0), and both
// phi planes equal phi0. The moments are rebuilt from the step-0 state: phi0 from its phi
// plane, U0 = sum g, rho0 = sum f, u0 = (sum c f) / rho0. Writes the node-local phi0 adjoint
// (phib_loc), the adjoint of grad phi0 (gbx, gby) and the adjoints of U0, rho0, u0.
struct InitAdjPtrs {
  const float* pops;     // state 0 (node-interleaved FP32 layout)
  const float* phi0;     // phi plane of state 0
  const float* pb;       // adjoint of the state-0 populations
  const float* Phib;     // adjoint of the state-0 phi plane
  const float* Psib;     // adjoint of the state-0 history plane
  float* phib_loc;
  float* gbx;
  float* gby;
  float* Ub;             // adjoints of the moments, [ny][pitch]
  float* rhob;
  float* uxb;
  float* uyb;
  double* partial;
};

template <bool FLOW>
__global__ void __launch_bounds__(256) adj_init_kernel(const Consts C, const InitAdjPtrs A) {
  const int x = blockIdx.x * 32 + (threadIdx.x & 31);
  const int y = blockIdx.y * 8 + (threadIdx.x >> 5);
  float part[kAdjParams] = {0.0f, 0.0f, 0.0f, 0.0f};
  if (x < C.nx && y < C.ny) {
    const long long Q = C.pstride, R = C.rstride, PI = C.pitch;
    const long long ip = (long long)y * R + x, iq = (long long)y * PI + x;
    const int xp = wrap_p(x + 1, C.nx), xm = wrap_m(x - 1, C.nx);
    const int yp = wrap_p(y + 1, C.ny), ym = wrap_m(y - 1, C.ny);
    auto P = [&](int xx, int yy) { return __ldg(A.phi0 + (long long)yy * PI + xx); };
    const float gx = kW1 * (P(xp, y) - P(xm, y)) + kW2 * ((P(xp, yp) - P(xm, yp)) +
                                                          (P(xp, ym) - P(xm, ym)));
    const float gy = kW1 * (P(x, yp) - P(x, ym)) + kW2 * ((P(xp, yp) - P(xp, ym)) +
                                                          (P(xm, yp) - P(xm, ym)));
    float gv[9], fv[9], hb[9], gbv[9], fbv[9];
    {
      float2 hg[9];
      load_hg_f32(A.pops, Q, ip, hg);
#pragma unroll
      for (int a = 0; a < 9; ++a) gv[a] = hg[a].y;
    }
    if (FLOW) {
      load_lattice_f32(A.pops + 18 * Q, Q, ip, fv);
    } else {
#pragma unroll
      for (int a = 0; a < 9; ++a) fv[a] = 0.0f;
    }
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      hb[a] = __ldg(A.pb + (PLANE_H + a) * Q + ip);
      gbv[a] = __ldg(A.pb + (PLANE_G + a) * Q + ip);
      fbv[a] = FLOW ? __ldg(A.pb + (PLANE_F + a) * Q + ip) : 0.0f;
    }
    const float U = sum9(gv);
    float rho = 1.0f, ux = 0.0f, uy = 0.0f;
    if (FLOW) {
      rho = sum9(fv);
      ux = sumcx9(fv) / rho;
      uy = sumcy9(fv) / rho;
    }
    // h_a = w_a (phi0 - Dphi3 c_a.N): node-local phi0 adjoint and the adjoint of N
    float phb = __ldg(A.Phib + iq) + __ldg(A.Psib + iq), Nxb = 0.0f, Nyb = 0.0f;
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      const float w = w_of(a);
      phb += w * hb[a];
      Nxb -= C.Dphi3 * w * hb[a] * (float)cx_of(a);
      Nyb -= C.Dphi3 * w * hb[a] * (float)cy_of(a);
    }
    float gxb = 0.0f, gyb = 0.0f;
    const float s2 = gx * gx + gy * gy;
    if (s2 > 1e-12f) {
      const float rinv = rsqrtf(s2);
      const float nx = gx * rinv, ny = gy * rinv;
      const float X2 = nx * nx, Y2 = ny * ny;
      const float cos6 = X2 * X2 * X2 - 15.0f * X2 * X2 * Y2 + 15.0f * X2 * Y2 * Y2 - Y2 * Y2 * Y2;
      const float Pp = 6.0f * X2 * X2 - 20.0f * X2 * Y2 + 6.0f * Y2 * Y2;
      const float sin6 = nx * ny * Pp;
      const float as = 1.0f + C.eps * cos6;
      const float t = C.kNkeps * as * sin6;
      const float tb = Nxb * gy - Nyb * gx;
      gyb += Nxb * t;
      gxb -= Nyb * t;
      const float as_b = tb * C.kNkeps * sin6;
      const float sin6_b = tb * C.kNkeps * as;
      part[ADJ_KN6EPS] += tb * as * sin6;
      const float cos6_b = as_b * C.eps;
      part[ADJ_EPS] += as_b * cos6;
      const float X2b = cos6_b * (3.0f * X2 * X2 - 30.0f * X2 * Y2 + 15.0f * Y2 * Y2) +
                        sin6_b * nx * ny * (12.0f * X2 - 20.0f * Y2);
      const float Y2b = cos6_b * (-15.0f * X2 * X2 + 30.0f * X2 * Y2 - 3.0f * Y2 * Y2) +
                        sin6_b * nx * ny * (-20.0f * X2 + 12.0f * Y2);
      const float nxb = sin6_b * ny * Pp + 2.0f * nx * X2b;
      const float nyb = sin6_b * nx * Pp + 2.0f * ny * Y2b;
      const float dn = nxb * nx + nyb * ny;
      gxb += rinv * (nxb - dn * nx);
      gyb += rinv * (nyb - dn * ny);
    }
    // g_a = w_a U0 (1 + 3 c_a.u0); f_a = w_a rho0 (1 + 3 cu + 4.5 cu^2 - 1.5 uu)
    float Ub = 0.0f, rhob = 0.0f, uxb = 0.0f, uyb = 0.0f;
    const float uu = ux * ux + uy * uy;
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      const float w = w_of(a);
      const float cu = cdot(a, ux, uy);
      Ub += gbv[a] * w * (1.0f + 3.0f * cu);
      float cub = gbv[a] * w * U * 3.0f;
      if (FLOW) {  // without the flow lattice u0 = 0 is not an input
        rhob += fbv[a] * w * (1.0f + 3.0f * cu + 4.5f * cu * cu - 1.5f * uu);
        cub += fbv[a] * w * rho * (3.0f + 9.0f * cu);
        uxb -= 3.0f * fbv[a] * w * rho * ux;
        uyb -= 3.0f * fbv[a] * w * rho * uy;
        uxb += cub * (float)cx_of(a);
        uyb += cub * (float)cy_of(a);
      }
    }
    A.phib_loc[iq] = phb;
    A.gbx[iq] = gxb;
    A.gby[iq] = gyb;
    A.Ub[iq] = Ub;
    A.rhob[iq] = rhob;
    A.uxb[iq] = uxb;
    A.uyb[iq] = uyb;
  }
  const int slot = blockIdx.y * gridDim.x + blockIdx.x;
  block_accumulate(part, A.partial + (long long)slot * kAdjParams);
}

// phi0 adjoint: the node-local part plus the transpose of the E4 stencil.
__global__ void __launch_bounds__(256) adj_gather_kernel(const Consts C,
                                                         const float* __restrict__ loc,
                                                         const float* __restrict__ gbx,
                                                         const float* __restrict__ gby,
                                                         float* __restrict__ out) {
  const int x = blockIdx.x * 32 + (threadIdx.x & 31);
  const int y = blockIdx.y * 8 + (threadIdx.x >> 5);
  if (x >= C.nx || y >= C.ny) return;
  const long long iq = (long long)y * C.pitch + x;
  out[iq] = __ldg(loc + iq) + e4_transpose(C, gbx, gby, x, y);
}

// Seed of the reverse sweep from dL/dphi_T and dL/dU_T ([ny][pitch] planes, either may be
// null): Phib = dL/dphi_T (phi_T is the phi plane), the g-population adjoints = dL/dU_T
// (U_T = sum g), every other adjoint zero.
template <bool FLOW>
__global__ void __launch_bounds__(256) adj_seed_kernel(const Consts C,
                                                       const float* __restrict__ phib_T,
                                                       const float* __restrict__ Ub_T,
                                                       float* __restrict__ pb,
                                                       float* __restrict__ Phib,
                                                       float* __restrict__ Psib) {
  const int x = blockIdx.x * 32 + (threadIdx.x & 31);
  const int y = blockIdx.y * 8 + (threadIdx.x >> 5);
  if (x >= C.nx || y >= C.ny) return;
  const long long Q = C.pstride, ip = (long long)y * C.rstride + x;
  const long long iq = (long long)y * C.pitch + x;
  const float u = Ub_T ? Ub_T[iq] : 0.0f;
#pragma unroll
  for (int a = 0; a < 9; ++a) {
    pb[(PLANE_H + a) * Q + ip] = 0.0f;
    pb[(PLANE_G + a) * Q + ip] = u;
    if (FLOW) pb[(PLANE_F + a) * Q + ip] = 0.0f;
  }
  Phib[iq] = phib_T ? phib_T[iq] : 0.0f;
  Psib[iq] = 0.0f;
}

}  // namespace lbmice
