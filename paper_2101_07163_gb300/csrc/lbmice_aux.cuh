// Auxiliary kernels: equilibrium initialisation from moment fields, the circular seed, moment
// export, checkpoint support and the FP64 diagnostic reductions.
#pragma once

#include "lbmice_device.cuh"

namespace lbmice {

// Circular seed (Sec. 3.1.2): phi = tanh((R0 - r) dx / (sqrt(2) W0)), U = U0, rho = 1,
// velocity = inlet velocity times the liquid fraction (1 - phi)/2. Fields are contiguous
// [ny][nx] doubles.
__global__ void seed_kernel(int nx, int ny, double cx, double cy, double R0, double U0,
                            double width, double ux_in, double uy_in, double* phi, double* U,
                            double* rho, double* ux, double* uy) {
  const int X = blockIdx.x * blockDim.x + threadIdx.x;
  const int Y = blockIdx.y * blockDim.y + threadIdx.y;
  if (X >= nx || Y >= ny) return;
  const long long i = (long long)Y * nx + X;
  const double dx = X - cx, dy = Y - cy;
  const double p = tanh((R0 - sqrt(dx * dx + dy * dy)) / width);
  phi[i] = p;
  U[i] = U0;
  if (rho) {  // flow fields (absent without the flow lattice)
    rho[i] = 1.0;
    const double liquid = 0.5 * (1.0 - p);
    ux[i] = ux_in * liquid;
    uy[i] = uy_in * liquid;
  }
}

// Populations at the equilibria of given moments, computed in double and stored in the
// storage type: h^eq (Eq. (e)) with the anisotropic flux of the gradient of phi, g^eq
// (Sec. 2.2.2), f^eq (Sec. 2.2.1), the gradient with the run's stencil and the anisotropy
// with its fold. The stored phi and its history both become sum h; with
// 16-bit storage U and rho become sum g and sum f.
template <bool FLOW, class S>
__global__ void equilibrium_kernel(const Consts C, double Dphi3, double eps, double kNkeps,
                                   const double* __restrict__ phi0,
                                   const double* __restrict__ U0,
                                   const double* __restrict__ rho0,
                                   const double* __restrict__ ux0,
                                   const double* __restrict__ uy0, void* pops,
                                   float* __restrict__ phi_cur, float* __restrict__ phi_prev,
                                   float* __restrict__ U_cur, float* __restrict__ rho_cur) {
  using ST = Storage<S>;
  const int X = blockIdx.x * blockDim.x + threadIdx.x;
  const int Y = blockIdx.y * blockDim.y + threadIdx.y;
  if (X >= C.nx || Y >= C.ny) return;
  auto P = [&](int x, int y) -> double {
    int gx, gy;
    if (axis_phi(x, C.nx, C.bc[0], C.bc[1], gx) && axis_phi(y, C.ny, C.bc[2], C.bc[3], gy))
      return phi0[(long long)gy * C.nx + gx];
    return -1.0;
  };
  const long long i = (long long)Y * C.nx + X;
  const double ph = phi0[i];
  double gx, gy;
  gradient_stencil<double>(C.stencil, [&](int dx, int dy) { return P(X + dx, Y + dy); }, gx,
                           gy);
  double as, Nx, Ny;
  aniso(gx, gy, eps, kNkeps, C.fold, as, Nx, Ny);
  const double U = U0[i];
  const double rho = rho0 ? rho0[i] : 1.0;
  const double ux = ux0 ? ux0[i] : 0.0;
  const double uy = uy0 ? uy0[i] : 0.0;
  const double uu = ux * ux + uy * uy;
  const long long o = (long long)Y * C.pitch + X;
  typename ST::T* pt = static_cast<typename ST::T*>(pops);
  const long long nd = (long long)Y * C.rstride + X;
  float hv[9], gv[9], fv[9];
#pragma unroll
  for (int a = 0; a < 9; ++a) {
    const double w = wd_of(a);
    hv[a] = (float)(w * (ph - Dphi3 * cdot(a, Nx, Ny)));
    const double cu = cdot(a, ux, uy);
    gv[a] = (float)(w * U * (1.0 + 3.0 * cu));
    fv[a] = (float)(w * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu));
  }
  const float s = sum9(hv);
  phi_cur[o] = s;
  phi_prev[o] = s;
  store9<S>(pt, 0, C.pstride, nd, s, hv);
  const float Ug = ST::DEV ? sum9(gv) : 0.0f;
  store9<S>(pt, 1, C.pstride, nd, Ug, gv);
  if (ST::DEV) U_cur[o] = Ug;
  if (FLOW) {
    const float rf = ST::DEV ? sum9(fv) : 0.0f;
    store9<S>(pt, 2, C.pstride, nd, rf, fv);
    if (ST::DEV) rho_cur[o] = rf;
  }
}

// Populations of lattice L (0 h, 1 g, 2 f) at node (X, Y), decoded to float.
template <class S>
__device__ __forceinline__ void node_lattice(const Consts& C, const void* pops, int L,
                                             const float* phi, const float* U,
                                             const float* rho, int X, int Y, float* out) {
  using ST = Storage<S>;
  const long long o = (long long)Y * C.pitch + X;
  float M = 0.0f;
  if (ST::DEV) M = L == 0 ? phi[o] : L == 1 ? U[o] : rho[o];
  load9<S>(static_cast<const typename ST::T*>(pops), L, C.pstride,
           (long long)Y * C.rstride + X, M, out);
}

// One decoded population plane (lattice L, direction a) into a contiguous [ny][nx] array.
template <class S>
__global__ void decode_plane_kernel(const Consts C, const void* pops, int L, int a,
                                    const float* phi, const float* U, const float* rho,
                                    float* __restrict__ out) {
  const int X = blockIdx.x * blockDim.x + threadIdx.x;
  const int Y = blockIdx.y * blockDim.y + threadIdx.y;
  if (X >= C.nx || Y >= C.ny) return;
  float v[9];
  node_lattice<S>(C, pops, L, phi, U, rho, X, Y, v);
  float r = v[0];
#pragma unroll
  for (int b = 1; b < 9; ++b) r = a == b ? v[b] : r;
  out[(long long)Y * C.nx + X] = r;
}

// Encode one lattice from 9 contiguous float planes [9][ny][nx]; its moment goes to M.
template <class S>
__global__ void encode_lattice_kernel(const Consts C, const float* __restrict__ planes, int L,
                                      void* pops, float* __restrict__ M) {
  const int X = blockIdx.x * blockDim.x + threadIdx.x;
  const int Y = blockIdx.y * blockDim.y + threadIdx.y;
  if (X >= C.nx || Y >= C.ny) return;
  const long long n = (long long)C.nx * C.ny, i = (long long)Y * C.nx + X;
  float v[9];
#pragma unroll
  for (int a = 0; a < 9; ++a) v[a] = planes[a * n + i];
  const float m = sum9(v);
  if (M) M[(long long)Y * C.pitch + X] = m;
  store9<S>(static_cast<typename Storage<S>::T*>(pops), L, C.pstride,
            (long long)Y * C.rstride + X, m, v);
}

// Moment of the current state into a contiguous [ny][nx] float array.
// which: 0 phi, 1 U, 2 rho, 3 u*_x, 4 u*_y, 5 phi history.
template <class S>
__global__ void moment_kernel(const Consts C, int which, int flow, const void* pops,
                              const float* __restrict__ phi, const float* __restrict__ phi_prev,
                              const float* __restrict__ U, const float* __restrict__ rho,
                              float* __restrict__ out) {
  const int X = blockIdx.x * blockDim.x + threadIdx.x;
  const int Y = blockIdx.y * blockDim.y + threadIdx.y;
  if (X >= C.nx || Y >= C.ny) return;
  const long long o = (long long)Y * C.pitch + X;
  float r = 0.0f;
  if (which == 0) {
    r = phi[o];
  } else if (which == 5) {
    r = phi_prev[o];
  } else if (which == 1) {
    float v[9];
    node_lattice<S>(C, pops, 1, phi, U, rho, X, Y, v);
    r = sum9(v);
  } else if (!flow) {
    r = which == 2 ? 1.0f : 0.0f;
  } else {
    float v[9];
    node_lattice<S>(C, pops, 2, phi, U, rho, X, Y, v);
    const float rh = sum9(v);
    if (which == 2) {
      r = rh;
    } else {
      const float ph = phi[o];
      const float onep = 1.0f + ph;
      const float k = C.kdrag * rh * onep * onep * (1.0f - ph);
      const float inv = 1.0f / (rh + 0.5f * k);
      const float sfac = 0.5f * (1.0f - ph);
      r = which == 3 ? sfac * (sumcx9(v) * inv) : sfac * (sumcy9(v) * inv);
    }
  }
  out[(long long)Y * C.nx + X] = r;
}

constexpr int kStatThreads = 256;
constexpr int kNStat = 5;

// Block-level partial sums in double: solid area, mass, vapour invariant, sum phi, count of
// non-finite nodes. One partial row per block; the final kernel adds rows in a fixed order,
// so the result does not depend on scheduling.
template <class S>
__global__ void __launch_bounds__(kStatThreads)
    stats_partial_kernel(const Consts C, int flow, double area_w, double half_Lsat,
                         const void* pops, const float* __restrict__ phi,
                         const float* __restrict__ phi_prev, const float* __restrict__ Um,
                         const float* __restrict__ rhom, double* __restrict__ partial) {
  double acc[kNStat] = {0.0, 0.0, 0.0, 0.0, 0.0};
  const long long n = (long long)C.nx * C.ny;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int Y = (int)(i / C.nx), X = (int)(i - (long long)Y * C.nx);
    const long long o = (long long)Y * C.pitch + X;
    const float ph = phi[o];
    float v[9];
    node_lattice<S>(C, pops, 1, phi, Um, rhom, X, Y, v);
    const float U = sum9(v);
    float rho = 1.0f;
    if (flow) {
      node_lattice<S>(C, pops, 2, phi, Um, rhom, X, Y, v);
      rho = sum9(v);
    }
    acc[0] += area_w * (1.0 + (double)ph);
    acc[1] += (double)rho;
    acc[2] += (double)U + half_Lsat * (double)phi_prev[o];
    acc[3] += (double)ph;
    acc[4] += (isfinite(ph) && isfinite(U) && isfinite(rho)) ? 0.0 : 1.0;
  }
  __shared__ double red[kNStat][kStatThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < kNStat; ++k) {
    double v = acc[k];
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if (lane == 0) red[k][warp] = v;
  }
  __syncthreads();
  if (threadIdx.x < kNStat) {
    double s = 0.0;
    for (int w = 0; w < kStatThreads / 32; ++w) s += red[threadIdx.x][w];
    partial[(long long)blockIdx.x * kNStat + threadIdx.x] = s;
  }
}

__global__ void stats_final_kernel(const double* __restrict__ partial, int nblocks,
                                   double* __restrict__ out) {
  if (threadIdx.x < kNStat) {
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += partial[(long long)b * kNStat + threadIdx.x];
    out[threadIdx.x] = s;
  }
}

// Tip positions: one warp per ray; the lanes evaluate 32 consecutive samples r = k step at a
// time and the first event along the ray (leaving the box [0, nx - 2] x [0, ny - 2], phi <= 0
// at the centre, or a crossing of phi from > 0 to <= 0) decides the result. phi is a
// [ny][pitch] plane; cs holds (cos, sin) of each ray's angle.
__device__ __forceinline__ double tip_bilinear(const float* __restrict__ phi, int pitch,
                                               double x, double y) {
  const int i = (int)x, j = (int)y;
  const double fx = x - i, fy = y - j;
  const float* p = phi + (long long)j * pitch + i;
  return ((double)p[0] * (1 - fx) + (double)p[1] * fx) * (1 - fy) +
         ((double)p[pitch] * (1 - fx) + (double)p[pitch + 1] * fx) * fy;
}

__global__ void tips_kernel(const float* __restrict__ phi, int nx, int ny, int pitch, double cx,
                            double cy, double step, int nrays, const double* __restrict__ cs,
                            double* __restrict__ radii) {
  const int ray = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (ray >= nrays) return;
  const double c = cs[2 * ray], s = cs[2 * ray + 1];
  double carry = 0.0;  // phi at the last sample of the previous group of 32
  for (long long base = 0;; base += 32) {
    const long long k = base + lane;
    const double r = (double)k * step;
    const double x = cx + r * c, y = cy + r * s;
    const bool outside = !(x >= 0.0 && y >= 0.0 && x <= nx - 2 && y <= ny - 2);
    const double v = outside ? 0.0 : tip_bilinear(phi, pitch, x, y);
    double pv = __shfl_up_sync(0xffffffffu, v, 1);
    if (lane == 0) pv = carry;
    const bool start_out = k == 0 && !outside && v <= 0.0;
    const bool cross = k > 0 && !outside && pv > 0.0 && v <= 0.0;
    const unsigned m = __ballot_sync(0xffffffffu, outside || start_out || cross);
    if (m) {
      if (lane == __ffs(m) - 1) {
        const double prev_r = (double)(k - 1) * step;
        radii[ray] = cross ? prev_r + (r - prev_r) * pv / (pv - v) : __longlong_as_double(0x7ff8000000000000LL);
      }
      return;
    }
    carry = __shfl_sync(0xffffffffu, v, 31);
  }
}

}  // namespace lbmice
