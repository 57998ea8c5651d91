// TEST INFRASTRUCTURE ONLY -- the plain FP64 CPU oracle of the coupled lattice-Boltzmann
// ice-crystal step of Tan, Hosseini, Seidel-Morgenstern, Thevenin and Lorenz,
// "Modeling ice crystal growth using the lattice Boltzmann method" (arXiv 2101.07163).
//
// Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may load this library.
// It shares no code, header, table or constant with the CUDA path; the two meet only at the
// seeded input fields (physical moments phi, U, rho, u) that both sides receive.
//
// The method is an explicit iteration, so this file is that iteration written step by step,
// in the paper's order and notation, with no blocking, fusion or reordering:
//   collide every node (Sec. 2.2.1 flow BGK + drag, Sec. 2.2.2 ADR for U, Sec. 2.2.3 Eq. (d)
//   for phi), then stream every population (pull), then rotate the phi history.
// All arithmetic is double, compiled with -O2 -ffp-contract=off and without -ffast-math.
// The node loops of a sweep may run on several host threads (OpenMP, rows split statically,
// orc_set_threads): every node writes only its own outputs and nothing is summed across
// nodes, so the results are bit-identical to one thread's.
//
// Readings of passages the paper leaves open (each is listed with its reason in the design
// notes of the repository):
//   R1  Eq. (a)/(e): the anisotropic flux |grad phi|^2 d(a_s^2)/d(grad phi) is taken with the
//       factor kappa_N/2 (kappa_N = 1: variational form a_s da_s/d(grad phi), the default).
//   R2  Isotropic gradient (Sec. 3.1.1, Table 1): weights w(1)=1/3, w(2)=1/12 already carry
//       the 1/c_s^2 factor, so the printed prefactor is not applied again.
//   R3  theta = arctan(n_y/n_x) enters only through cos(6 theta), sin(6 theta), evaluated as
//       polynomials of the unit normal (pi-periodic, so the quadrant does not matter).
//   R4  |grad phi|^2 <= 1e-12 (lattice units): a_s = 1, no anisotropic flux.
//   R5  a_s^2 in Eq. (d) is evaluated at the collision node x.
//   R6  h_alpha(x + c_alpha, t) in Eq. (d) is the stored pre-collision population at time t;
//       the update is applied in pull form at the destination y = x + c_alpha.
//   R7  d(phi)/dt in the U source (Sec. 2.2.2) is the backward difference at the collision
//       node, with phi^{-1} = phi^0.
//   R8  q(phi) = 1 - phi as printed, clamped to [0, 2].
//   R9  The velocity in g^eq is u* = (1 - phi)/2 u.
//   R10 Drag enters through Guo forcing; u = j / (rho + k/2), u* = (1 - phi)/2 u is used in
//       f^eq and in F = -k u*, with k = h rho nu (1+phi)^2 (1-phi) / (4 W0^2), h = 2.757.
//   R11 D2Q9 with second-order Hermite equilibria for all three lattices; c_s^2 = 1/3.
//   R12 Unit conversion: diffusivities scale with dt/dx^2, the anisotropic flux with dt/dx.
//   R13 Initial populations are the equilibria of the given moments.
//   R14 All couplings use time-n moments (Jacobi).
//   R15 Boundary ghosts: periodic wrap; zero-gradient outlet = copy of the adjacent node;
//       free-slip = mirror image of the adjacent node; inlet = equilibrium at the inlet state.
//   R18 lambda, when not given, is the beta = 0 choice tau0 D / (a2 W0^2), a2 = 0.6267.
//   R21 E2 is the central difference; E6/E8 use the shell weights of Table 1, which (as R2)
//       already carry 1/c_s^2: E6 w(1,2,4) = 4/15, 1/10, 1/120; E8 w(1,2,4,5,8) = 4/21,
//       4/45, 1/60, 2/315, 1/5040.
//   R22 The four-fold system (Sec. 3.1.2) uses the same anisotropy with k = 4:
//       a_s = 1 + eps cos(4 theta), flux kappa_N a_s 4 eps sin(4 theta) (g_y, -g_x).
// (R19, R20, R23 and R24 concern the workloads and the GPU storage, not this arithmetic.)
// Parity is pinned by tests/test_oracle_pins.py, tests/test_oracle_grad_pins.py and
// tests/test_oracle_variant_pins.py (closed forms, invariants, symmetries,
// brute force); no function here is unpinned.

#include <omp.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

namespace {

// ---------------------------------------------------------------------------------------
// D2Q9 velocity set (paper Sec. 2.2; the stencil is not named there, R11).
//   alpha : 0      1      2      3       4       5      6       7        8
//   c     : (0,0) (1,0)  (0,1)  (-1,0)  (0,-1)  (1,1)  (-1,1)  (-1,-1)  (1,-1)
// ---------------------------------------------------------------------------------------
const int kCx[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
const int kCy[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
const double kW[9] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0, 1.0 / 9.0,
                      1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
// alpha of the velocity reflected across a vertical line (cx -> -cx) / horizontal line.
const int kMirX[9] = {0, 3, 2, 1, 4, 6, 5, 8, 7};
const int kMirY[9] = {0, 1, 4, 3, 2, 8, 7, 6, 5};

const double kCs2 = 1.0 / 3.0;   // lattice sound speed squared
const double kA2 = 0.6267;       // Sec. 2.1, a2 for g(phi) = phi - 2phi^3/3 + phi^5/5
const double kHdrag = 2.757;     // Sec. 2.2.1, dimensionless drag constant h
const double kGradEps = 1e-12;   // R4

enum { BC_PERIODIC = 0, BC_INLET = 1, BC_OUTLET = 2, BC_FREESLIP = 3 };

// Symmetric sum over the nine directions: rest, the four axis pairs, the four diagonal
// pairs. Every reflection of the square maps this tree onto itself, so a mirror-symmetric
// state gives bit-identical sums at mirror nodes.
template <class T>
T sum9(const T v[9]) {
  return v[0] + (((v[1] + v[3]) + (v[2] + v[4])) + ((v[5] + v[7]) + (v[6] + v[8])));
}
// First moments with the same pairing: sum c_x v, sum c_y v.
template <class T>
T sumcx9(const T v[9]) {
  return (v[1] - v[3]) + ((v[5] - v[7]) + (v[8] - v[6]));
}
template <class T>
T sumcy9(const T v[9]) {
  return (v[2] - v[4]) + ((v[5] - v[7]) + (v[6] - v[8]));
}

}  // namespace

extern "C" {

// Physical parameters of one run (Sec. 2.1-2.2 and Sec. 3). W0, tau0, dx, dt, D in one
// consistent unit system; u_in and nu are in lattice units (dx/dt and dx^2/dt).
typedef struct {
  int32_t nx, ny;
  double dx, dt, W0, tau0;
  double D, lambda, L_sat, eps, kappa_N;
  double U_in, u_in, nu;
  int32_t bc[4];  // faces -x, +x, -y, +y
  int32_t flow;   // 1: flow lattice f is evolved; 0: fluid at rest, f absent
  int32_t stencil;  // gradient of Sec. 3.1.1: 2 (central difference), 4, 6, 8 (Table 1); 0 = 4
  int32_t fold;     // anisotropy symmetry: 6 (ice, Sec. 2.1) or 4 (validation case); 0 = 6
} orc_params;

}  // extern "C"

namespace {

// Lattice constants derived from the physical parameters (R12).
struct Derived {
  double Dphi;     // (W0^2/tau0) dt/dx^2: lattice diffusivity of phi
  double dt_tau0;  // dt/tau0: weight of the phase-field source
  double Dlat;     // D dt/dx^2: lattice vapour diffusivity
  double Wlat;     // W0/dx: interface width in cells
  double lambda;   // coupling constant (beta = 0 choice, Sec. 2.1, when not given)
  double tau_f;    // flow relaxation time nu/c_s^2 + 1/2
};

template <class T>
struct Oracle {
  orc_params p;
  Derived d;
  // The parameters the gradient of the method is taken with respect to, in the scalar type
  // of the run (for T = double they are exactly p.eps, d.Dlat and d.lambda).
  T eps = T(0.0), Dlat = T(0.0), lambda = T(0.0);
  // When set, the values (not the derivatives) of phi = sum h used by the next collision are
  // taken from this [ny][nx] array: a gradient run differentiating along given states.
  const double* phi_force = nullptr;
  int nx = 0, ny = 0;
  size_t n = 0;
  // Pre-collision populations at time t, one array per direction, node index y*nx + x.
  std::vector<T> f[9], g[9], h[9];
  std::vector<T> phi_prev;  // phi at time t - 1 (R7)
  // Per-step work arrays: post-collision populations and a_s^2 at every node.
  std::vector<T> fs[9], gs[9], hs[9], as2;
  std::vector<T> fn[9], gn[9], hn[9];
  int64_t steps = 0;

  size_t at(int x, int y) const { return (size_t)y * nx + x; }
};

// Ghost resolution (R15). A coordinate outside the grid is mapped through the face rules
// of x and then y. kind 0: the ghost carries the state of node (mx, my), with directions
// reflected where a free-slip face was crossed; kind 1: the ghost is an inlet node.
struct Ghost {
  int kind;
  int mx, my;
  bool mirx, miry;
  int inlet_face;
};

Ghost resolve(const orc_params& p, int x, int y) {
  Ghost r{0, x, y, false, false, -1};
  const int nx = p.nx, ny = p.ny;
  if (x < 0 || x >= nx) {
    const int face = x < 0 ? 0 : 1;
    switch (p.bc[face]) {
      case BC_PERIODIC: r.mx = x < 0 ? x + nx : x - nx; break;
      case BC_OUTLET: r.mx = x < 0 ? 0 : nx - 1; break;
      case BC_FREESLIP: r.mx = x < 0 ? -1 - x : 2 * nx - 1 - x; r.mirx = true; break;
      default: r.mx = x < 0 ? 0 : nx - 1; r.kind = 1; r.inlet_face = face; break;
    }
  }
  if (y < 0 || y >= ny) {
    const int face = y < 0 ? 2 : 3;
    switch (p.bc[face]) {
      case BC_PERIODIC: r.my = y < 0 ? y + ny : y - ny; break;
      case BC_OUTLET: r.my = y < 0 ? 0 : ny - 1; break;
      case BC_FREESLIP: r.my = y < 0 ? -1 - y : 2 * ny - 1 - y; r.miry = true; break;
      default:
        r.my = y < 0 ? 0 : ny - 1;
        if (r.kind == 0) { r.kind = 1; r.inlet_face = face; }
        break;
    }
  }
  return r;
}

// Inlet velocity: magnitude u_in along the inward normal of the inlet face.
void inlet_velocity(const orc_params& p, int face, double* ux, double* uy) {
  *ux = 0.0; *uy = 0.0;
  if (face == 0) *ux = p.u_in;
  if (face == 1) *ux = -p.u_in;
  if (face == 2) *uy = p.u_in;
  if (face == 3) *uy = -p.u_in;
}

}  // namespace

namespace {

// ---------------------------------------------------------------------------------------
// Isotropic first derivative, E4 stencil (Sec. 3.1.1 and Table 1): the gradient is the sum
// over the neighbour shells of w(|c|^2) phi(x + c) c with w(1) = 1/3, w(2) = 1/12 (R2).
// On D2Q9 the |c|^2 = 1 shell is the four axis neighbours and |c|^2 = 2 the four diagonal
// ones. The eight terms are grouped by opposite neighbours so that mirror images of a field
// give gradients that are exact mirror images. Result in lattice units (per cell).
// ---------------------------------------------------------------------------------------
const double kWg1 = 1.0 / 3.0;
const double kWg2 = 1.0 / 12.0;

template <class T>
void grad_e4(T pE, T pW, T pN, T pS, T pNE, T pNW, T pSE, T pSW, T* gx, T* gy) {
  *gx = kWg1 * (pE - pW) + kWg2 * ((pNE - pNW) + (pSE - pSW));
  *gy = kWg1 * (pN - pS) + kWg2 * ((pNE - pSE) + (pNW - pSW));
}

// The gradient with the stencil of the run (Sec. 3.1.1): E2 is the central difference; E4, E6
// and E8 sum w(|c|^2) phi(x + c) c over the neighbour shells of Table 1 (|c|^2 = 1, 2, 4, 5,
// 8), with the weights as printed (they carry the 1/c_s^2, R2). P(dx, dy) is phi at the
// offset. Every shell is a sum of differences of opposite neighbours, grouped so that a
// mirrored field gives the exactly mirrored gradient.
int stencil_of(const orc_params& p) { return p.stencil == 0 ? 4 : p.stencil; }
int fold_of(const orc_params& p) { return p.fold == 0 ? 6 : p.fold; }

template <class T, class F>
void gradient_stencil(int stencil, F P, T* gx, T* gy) {
  if (stencil == 2) {
    *gx = 0.5 * (P(1, 0) - P(-1, 0));
    *gy = 0.5 * (P(0, 1) - P(0, -1));
    return;
  }
  double w1 = kWg1, w2 = kWg2, w4 = 0.0, w5 = 0.0, w8 = 0.0;
  if (stencil == 6) {
    w1 = 4.0 / 15.0; w2 = 1.0 / 10.0; w4 = 1.0 / 120.0;
  } else if (stencil == 8) {
    w1 = 4.0 / 21.0; w2 = 4.0 / 45.0; w4 = 1.0 / 60.0; w5 = 2.0 / 315.0; w8 = 1.0 / 5040.0;
  }
  T ax = w1 * (P(1, 0) - P(-1, 0)) + w2 * ((P(1, 1) - P(-1, 1)) + (P(1, -1) - P(-1, -1)));
  T ay = w1 * (P(0, 1) - P(0, -1)) + w2 * ((P(1, 1) - P(1, -1)) + (P(-1, 1) - P(-1, -1)));
  if (stencil >= 6) {
    ax = ax + (2.0 * w4) * (P(2, 0) - P(-2, 0));
    ay = ay + (2.0 * w4) * (P(0, 2) - P(0, -2));
  }
  if (stencil == 8) {
    ax = ax + w5 * (((P(1, 2) - P(-1, 2)) + (P(1, -2) - P(-1, -2))) +
                    2.0 * ((P(2, 1) - P(-2, 1)) + (P(2, -1) - P(-2, -1))));
    ay = ay + w5 * (2.0 * ((P(1, 2) - P(1, -2)) + (P(-1, 2) - P(-1, -2))) +
                    ((P(2, 1) - P(2, -1)) + (P(-2, 1) - P(-2, -1))));
    ax = ax + (2.0 * w8) * ((P(2, 2) - P(-2, 2)) + (P(2, -2) - P(-2, -2)));
    ay = ay + (2.0 * w8) * ((P(2, 2) - P(2, -2)) + (P(-2, 2) - P(-2, -2)));
  }
  *gx = ax;
  *gy = ay;
}

// ---------------------------------------------------------------------------------------
// Six-fold anisotropy (Sec. 2.1): a_s(n) = 1 + eps cos(6 theta), theta the angle of the
// interface normal n = -grad phi / |grad phi| (R3, R4), and the anisotropic flux of Eq. (a)
// and Eq. (e), N = (kappa_N / 2) |grad phi|^2 d(a_s^2)/d(grad phi) (R1). Differentiating
// a_s through theta = atan2(g_y, g_x) gives |g|^2 da_s/dg = 6 eps sin(6 theta) (g_y, -g_x),
// so N = kappa_N a_s 6 eps sin(6 theta) (g_y, -g_x). N is linear in g and carries its units.
// ---------------------------------------------------------------------------------------
template <class T, class P>
void anisotropy(T gx, T gy, P eps, double kappa_N, int fold, T* as, T* Nx, T* Ny) {
  const T s = gx * gx + gy * gy;
  if (!(s > kGradEps)) {
    *as = T(1.0);
    *Nx = T(0.0);
    *Ny = T(0.0);
    return;
  }
  using std::sqrt;
  const T r = sqrt(s);
  const T nx = gx / r;
  const T ny = gy / r;
  const T X = nx * nx;
  const T Y = ny * ny;
  if (fold == 4) {
    // the four-fold validation case: cos(4 theta), sin(4 theta) from (n_x + i n_y)^4, and
    // |g|^2 da_s/dg = 4 eps sin(4 theta) (g_y, -g_x)
    const T cos4 = X * X - 6.0 * X * Y + Y * Y;
    const T sin4 = 4.0 * nx * ny * (X - Y);
    *as = 1.0 + eps * cos4;
    const T t4 = kappa_N * (*as) * (4.0 * eps) * sin4;
    *Nx = t4 * gy;
    *Ny = -(t4 * gx);
    return;
  }
  // cos(6 theta) and sin(6 theta) as the real and imaginary parts of (n_x + i n_y)^6.
  const T cos6 = X * X * X - 15.0 * X * X * Y + 15.0 * X * Y * Y - Y * Y * Y;
  const T sin6 = nx * ny * (6.0 * X * X - 20.0 * X * Y + 6.0 * Y * Y);
  *as = 1.0 + eps * cos6;
  const T t = kappa_N * (*as) * (6.0 * eps) * sin6;
  *Nx = t * gy;
  *Ny = -(t * gx);
}

// Second-order Hermite equilibrium of the flow lattice (Sec. 2.2.1):
// f^eq = w rho (1 + c.u / c_s^2 + (c.u)^2 / (2 c_s^4) - u.u / (2 c_s^2)).
template <class T>
T feq(int a, T rho, T ux, T uy) {
  const T cu = double(kCx[a]) * ux + double(kCy[a]) * uy;
  const T uu = ux * ux + uy * uy;
  return kW[a] * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
}

// Equilibrium of the vapour lattice (Sec. 2.2.2): g^eq = w U (1 + c.u / c_s^2).
template <class T>
T geq(int a, T U, T ux, T uy) {
  const T cu = double(kCx[a]) * ux + double(kCy[a]) * uy;
  return kW[a] * U * (1.0 + 3.0 * cu);
}

// Equilibrium of the phase-field lattice, Eq. (e), in lattice units (R12):
// h^eq = w (phi - (1/c_s^2) c.N (W0^2/tau0) dt/dx^2), N from the lattice-unit gradient.
template <class T>
T heq(int a, T phi, T Nx, T Ny, double Dphi) {
  const T cN = double(kCx[a]) * Nx + double(kCy[a]) * Ny;
  return kW[a] * (phi - 3.0 * Dphi * cN);
}

bool derive(const orc_params& p, Derived* d) {
  if (p.nx < 1 || p.ny < 1) return false;
  if (!(p.dx > 0) || !(p.dt > 0) || !(p.W0 > 0) || !(p.tau0 > 0) || !(p.D >= 0)) return false;
  for (int f = 0; f < 4; ++f)
    if (p.bc[f] < BC_PERIODIC || p.bc[f] > BC_FREESLIP) return false;
  if ((p.bc[0] == BC_PERIODIC) != (p.bc[1] == BC_PERIODIC)) return false;
  if ((p.bc[2] == BC_PERIODIC) != (p.bc[3] == BC_PERIODIC)) return false;
  if (p.stencil != 0 && p.stencil != 2 && p.stencil != 4 && p.stencil != 6 && p.stencil != 8)
    return false;
  if (p.fold != 0 && p.fold != 4 && p.fold != 6) return false;
  d->Dphi = (p.W0 * p.W0 / p.tau0) * p.dt / (p.dx * p.dx);
  d->dt_tau0 = p.dt / p.tau0;
  d->Dlat = p.D * p.dt / (p.dx * p.dx);
  d->Wlat = p.W0 / p.dx;
  // Sec. 2.1: beta = 0 when tau0 = a2 lambda W0^2 / D, i.e. lambda = tau0 D / (a2 W0^2).
  d->lambda = p.lambda > 0 ? p.lambda : p.tau0 * p.D / (kA2 * p.W0 * p.W0);
  // Sec. 2.2.1: tau = nu / c_s^2 + 1/2 (nu in lattice units).
  d->tau_f = p.nu / kCs2 + 0.5;
  if (p.flow && !(d->tau_f > 0.5)) return false;
  return true;
}

template <class T>
void alloc(Oracle<T>* o) {
  const size_t n = o->n;
  for (int a = 0; a < 9; ++a) {
    o->g[a].assign(n, T(0.0)); o->h[a].assign(n, T(0.0));
    o->gs[a].assign(n, T(0.0)); o->hs[a].assign(n, T(0.0));
    o->gn[a].assign(n, T(0.0)); o->hn[a].assign(n, T(0.0));
    if (o->p.flow) {
      o->f[a].assign(n, T(0.0)); o->fs[a].assign(n, T(0.0)); o->fn[a].assign(n, T(0.0));
    }
  }
  o->phi_prev.assign(n, T(0.0));
  o->as2.assign(n, T(1.0));
}

// Zeroth moment of h at every node: phi = sum_alpha h_alpha (Sec. 2.2.3).
template <class T>
void phi_field(const Oracle<T>& o, std::vector<T>* phi) {
  phi->resize(o.n);
#pragma omp parallel for schedule(static)
  for (long long i = 0; i < (long long)o.n; ++i) {
    T v[9];
    for (int a = 0; a < 9; ++a) v[a] = o.h[a][i];
    (*phi)[i] = sum9(v);
  }
}

// phi at any coordinate, ghosts resolved by the face rules (inlet ghosts hold vapour, -1).
template <class T>
T phi_ghost(const Oracle<T>& o, const std::vector<T>& phi, int x, int y) {
  if (x >= 0 && x < o.nx && y >= 0 && y < o.ny) return phi[o.at(x, y)];
  const Ghost r = resolve(o.p, x, y);
  if (r.kind == 1) return T(-1.0);
  return phi[o.at(r.mx, r.my)];
}

template <class T>
void gradient_at(const Oracle<T>& o, const std::vector<T>& phi, int x, int y, T* gx, T* gy) {
  auto P = [&](int dx, int dy) { return phi_ghost(o, phi, x + dx, y + dy); };
  gradient_stencil(stencil_of(o.p), P, gx, gy);
}

// Fluid velocity of a node (R10): u = j / (rho + k/2) and the solid-damped u* = (1-phi)/2 u.
template <class T>
void flow_velocity(const Oracle<T>& o, T phi, T rho, T jx, T jy, T* k, T* usx, T* usy) {
  const double nu = o.p.nu;
  *k = kHdrag * rho * nu * (1.0 + phi) * (1.0 + phi) * (1.0 - phi) /
       (4.0 * o.d.Wlat * o.d.Wlat);
  const T ux = jx / (rho + 0.5 * (*k));
  const T uy = jy / (rho + 0.5 * (*k));
  const T sfac = 0.5 * (1.0 - phi);
  *usx = sfac * ux;
  *usy = sfac * uy;
}

}  // namespace

namespace {

// ---------------------------------------------------------------------------------------
// Collision of every node (the right-hand sides of the three LB equations of Sec. 2.2),
// from the time-n state (R14). Fills fs, gs, hs (post-collision populations) and as2.
// ---------------------------------------------------------------------------------------
inline void set_value(double& x, double v) { x = v; }

template <class T>
void collide(Oracle<T>* o) {
  const orc_params& p = o->p;
  const Derived& d = o->d;
  std::vector<T> phi;
  phi_field(*o, &phi);
  if (o->phi_force)
    for (size_t i = 0; i < o->n; ++i) set_value(phi[i], o->phi_force[i]);
#pragma omp parallel for schedule(static)
  for (int y = 0; y < o->ny; ++y) {
    for (int x = 0; x < o->nx; ++x) {
      const size_t i = o->at(x, y);
      T hv[9], gv[9], fv[9];
      for (int a = 0; a < 9; ++a) { hv[a] = o->h[a][i]; gv[a] = o->g[a][i]; }
      // Moments (Sec. 2.2.2: U = sum g; Sec. 2.2.3: phi = sum h; Sec. 2.2.1: rho, rho u).
      const T ph = phi[i];
      const T U = sum9(gv);
      T rho = T(1.0), jx = T(0.0), jy = T(0.0);
      if (p.flow) {
        for (int a = 0; a < 9; ++a) fv[a] = o->f[a][i];
        rho = sum9(fv);
        jx = sumcx9(fv);
        jy = sumcy9(fv);
      }
      // Gradient, anisotropy and the phase-field relaxation time (Sec. 2.2.3).
      T gx, gy, as, Nx, Ny;
      gradient_at(*o, phi, x, y, &gx, &gy);
      anisotropy(gx, gy, o->eps, p.kappa_N, fold_of(p), &as, &Nx, &Ny);
      const T a2 = as * as;
      const T eta = 3.0 * a2 * d.Dphi + 0.5;
      const T Qphi = ph - ph * ph * ph + o->lambda * U * (1.0 - ph * ph) * (1.0 - ph * ph);
      o->as2[i] = a2;
      for (int a = 0; a < 9; ++a) {
        const T he = heq(a, ph, Nx, Ny, d.Dphi);
        o->hs[a][i] = hv[a] - (hv[a] - he) / eta + kW[a] * Qphi * d.dt_tau0;
      }
      // Fluid velocity with solid damping and drag (Sec. 2.2.1, R10).
      T k = T(0.0), usx = T(0.0), usy = T(0.0);
      if (p.flow) flow_velocity(*o, ph, rho, jx, jy, &k, &usx, &usy);
      // Vapour: q(phi), tau_g, g^eq with u*, source -w L_sat/2 dphi/dt (Sec. 2.2.2, R7-R9).
      T q = 1.0 - ph;
      if (q < 0.0) q = T(0.0);
      if (q > 2.0) q = T(2.0);
      const T tau_g = 3.0 * o->Dlat * q + 0.5;
      const T src = -0.5 * p.L_sat * (ph - o->phi_prev[i]);  // (dphi/dt) * dt
      for (int a = 0; a < 9; ++a) {
        const T ge = geq(a, U, usx, usy);
        o->gs[a][i] = gv[a] - (gv[a] - ge) / tau_g + kW[a] * src;
      }
      // Flow: BGK towards f^eq(rho, u*) plus Guo's forcing of F = -k u*.
      if (p.flow) {
        const T Fx = -k * usx;
        const T Fy = -k * usy;
        const T uF = usx * Fx + usy * Fy;
        const double pref = 1.0 - 0.5 / d.tau_f;
        for (int a = 0; a < 9; ++a) {
          const T fe = feq(a, rho, usx, usy);
          const T cu = double(kCx[a]) * usx + double(kCy[a]) * usy;
          const T cF = double(kCx[a]) * Fx + double(kCy[a]) * Fy;
          const T force = pref * kW[a] * (3.0 * (cF - uF) + 9.0 * cu * cF);
          o->fs[a][i] = fv[a] - (fv[a] - fe) / d.tau_f + force;
        }
      }
    }
  }
}

// Post-collision value carried by direction a out of source coordinate (sx, sy), which may
// be a ghost (R15). Returns f*, g*, h* and a_s^2 of that source.
template <class T>
void source_values(const Oracle<T>& o, int a, int sx, int sy, T* fsv, T* gsv, T* hsv, T* a2) {
  if (sx >= 0 && sx < o.nx && sy >= 0 && sy < o.ny) {
    const size_t s = o.at(sx, sy);
    *fsv = o.p.flow ? o.fs[a][s] : T(0.0);
    *gsv = o.gs[a][s];
    *hsv = o.hs[a][s];
    *a2 = o.as2[s];
    return;
  }
  const Ghost r = resolve(o.p, sx, sy);
  const size_t m = o.at(r.mx, r.my);
  if (r.kind == 0) {
    int am = a;
    if (r.mirx) am = kMirX[am];
    if (r.miry) am = kMirY[am];
    *fsv = o.p.flow ? o.fs[am][m] : T(0.0);
    *gsv = o.gs[am][m];
    *hsv = o.hs[am][m];
    *a2 = o.as2[m];
    return;
  }
  // Inlet ghost: vapour (phi = -1) at the equilibrium of the inlet state; the density is
  // that of the adjacent node, the velocity u_in along the inward normal; a_s = 1.
  double ux, uy;
  inlet_velocity(o.p, r.inlet_face, &ux, &uy);
  T rho_adj = T(1.0);
  if (o.p.flow) {
    T fv[9];
    for (int b = 0; b < 9; ++b) fv[b] = o.f[b][m];
    rho_adj = sum9(fv);
  }
  *fsv = o.p.flow ? feq(a, rho_adj, T(ux), T(uy)) : T(0.0);
  *gsv = geq(a, T(o.p.U_in), T(ux), T(uy));
  *hsv = T(-kW[a]);
  *a2 = T(1.0);
}

// Streaming (pull form). Flow and vapour: f_a(y, t+1) = f*_a(y - c_a). Phase field, Eq. (d)
// at x = y - c_a solved for the new population (R5, R6):
//   h_a(y, t+1) = h_a(y, t) + [h*_a(x) - h_a(y, t)] / a_s^2(x).
template <class T>
void stream(Oracle<T>* o) {
#pragma omp parallel for schedule(static)
  for (int y = 0; y < o->ny; ++y) {
    for (int x = 0; x < o->nx; ++x) {
      const size_t i = o->at(x, y);
      for (int a = 0; a < 9; ++a) {
        T fsv, gsv, hsv, a2;
        source_values(*o, a, x - kCx[a], y - kCy[a], &fsv, &gsv, &hsv, &a2);
        if (o->p.flow) o->fn[a][i] = fsv;
        o->gn[a][i] = gsv;
        const T hold = o->h[a][i];
        o->hn[a][i] = hold + (hsv - hold) / a2;
      }
    }
  }
}

template <class T>
void step_once(Oracle<T>* o) {
  collide(o);
  std::vector<T> phi;
  phi_field(*o, &phi);  // phi^n becomes the history of the next step (R7)
  stream(o);
  for (int a = 0; a < 9; ++a) {
    o->h[a].swap(o->hn[a]);
    o->g[a].swap(o->gn[a]);
    if (o->p.flow) o->f[a].swap(o->fn[a]);
  }
  o->phi_prev.swap(phi);
  o->steps += 1;
}

// Initial populations: equilibria of the given moments (R13); phi^{-1} = phi^0 (R7).
// rho, ux, uy may be empty (fluid at rest); without the flow lattice they are ignored.
template <class T>
void init_fields_t(Oracle<T>* o, const std::vector<T>& phi, const std::vector<T>& U,
                   const std::vector<T>& rho0, const std::vector<T>& ux0,
                   const std::vector<T>& uy0) {
  for (int y = 0; y < o->ny; ++y) {
    for (int x = 0; x < o->nx; ++x) {
      const size_t i = o->at(x, y);
      T gx, gy, as, Nx, Ny;
      gradient_at(*o, phi, x, y, &gx, &gy);
      anisotropy(gx, gy, o->eps, o->p.kappa_N, fold_of(o->p), &as, &Nx, &Ny);
      // without the flow lattice the fluid is at rest (rho = 1, u = 0)
      const bool fl = o->p.flow != 0;
      const T rho = (fl && !rho0.empty()) ? rho0[i] : T(1.0);
      const T ux = (fl && !ux0.empty()) ? ux0[i] : T(0.0);
      const T uy = (fl && !uy0.empty()) ? uy0[i] : T(0.0);
      for (int a = 0; a < 9; ++a) {
        o->h[a][i] = heq(a, phi[i], Nx, Ny, o->d.Dphi);
        o->g[a][i] = geq(a, U[i], ux, uy);
        if (o->p.flow) o->f[a][i] = feq(a, rho, ux, uy);
      }
    }
  }
  phi_field(*o, &o->phi_prev);
  o->steps = 0;
}

template <class T>
void init_fields(Oracle<T>* o, const double* phi0, const double* U0, const double* rho0,
                 const double* ux0, const double* uy0) {
  auto vec = [&](const double* a) {
    std::vector<T> v;
    if (a) v.assign(a, a + o->n);
    return v;
  };
  init_fields_t(o, vec(phi0), vec(U0), vec(rho0), vec(ux0), vec(uy0));
}

// Moments of the current state. which: 0 phi, 1 U, 2 rho, 3 u*_x, 4 u*_y, 5 phi history.
template <class T>
void get_field(const Oracle<T>& o, int which, double* out) {
  T v[9], fv[9];
  for (size_t i = 0; i < o.n; ++i) {
    T r = T(0.0);
    if (which == 0) {
      for (int a = 0; a < 9; ++a) v[a] = o.h[a][i];
      r = sum9(v);
    } else if (which == 1) {
      for (int a = 0; a < 9; ++a) v[a] = o.g[a][i];
      r = sum9(v);
    } else if (which == 5) {
      r = o.phi_prev[i];
    } else if (!o.p.flow) {
      r = which == 2 ? T(1.0) : T(0.0);
    } else {
      for (int a = 0; a < 9; ++a) { fv[a] = o.f[a][i]; v[a] = o.h[a][i]; }
      const T rho = sum9(fv);
      if (which == 2) {
        r = rho;
      } else {
        T k, usx, usy;
        flow_velocity(o, sum9(v), rho, sumcx9(fv), sumcy9(fv), &k, &usx, &usy);
        r = which == 3 ? usx : usy;
      }
    }
    out[i] = double(r);
  }
}

}  // namespace

// ---------------------------------------------------------------------------------------
// Forward-mode dual numbers: a value and N directional derivatives, carried through the same
// templated iteration as the double oracle, so a run yields the exact derivatives of the
// discrete map (up to rounding) with respect to the seeded directions. The clamp of q (R8)
// and the |grad phi| threshold (R4) are differentiated as the branch taken (zero slope
// beyond the clamp, a_s = 1 below the threshold).
// ---------------------------------------------------------------------------------------
namespace {

template <int N>
struct Dual {
  double v = 0.0;
  double d[N] = {};
  Dual() = default;
  Dual(double x) : v(x) {}  // constants carry no derivative
  explicit operator double() const { return v; }
};

template <int N> Dual<N> operator-(const Dual<N>& a) {
  Dual<N> r(-a.v);
  for (int i = 0; i < N; ++i) r.d[i] = -a.d[i];
  return r;
}
template <int N> Dual<N> operator+(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r(a.v + b.v);
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] + b.d[i];
  return r;
}
template <int N> Dual<N> operator-(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r(a.v - b.v);
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] - b.d[i];
  return r;
}
// product rule: (ab)' = a'b + ab'
template <int N> Dual<N> operator*(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r(a.v * b.v);
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
  return r;
}
// quotient rule: (a/b)' = (a'b - ab') / b^2, written as (a' - (a/b) b') / b
template <int N> Dual<N> operator/(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r(a.v / b.v);
  for (int i = 0; i < N; ++i) r.d[i] = (a.d[i] - r.v * b.d[i]) / b.v;
  return r;
}
template <int N> Dual<N> operator+(const Dual<N>& a, double b) { return a + Dual<N>(b); }
template <int N> Dual<N> operator+(double a, const Dual<N>& b) { return Dual<N>(a) + b; }
template <int N> Dual<N> operator-(const Dual<N>& a, double b) { return a - Dual<N>(b); }
template <int N> Dual<N> operator-(double a, const Dual<N>& b) { return Dual<N>(a) - b; }
template <int N> Dual<N> operator*(const Dual<N>& a, double b) { return a * Dual<N>(b); }
template <int N> Dual<N> operator*(double a, const Dual<N>& b) { return Dual<N>(a) * b; }
template <int N> Dual<N> operator/(const Dual<N>& a, double b) { return a / Dual<N>(b); }
template <int N> Dual<N> operator/(double a, const Dual<N>& b) { return Dual<N>(a) / b; }
template <int N> bool operator>(const Dual<N>& a, double b) { return a.v > b; }
template <int N> void set_value(Dual<N>& x, double v) { x.v = v; }
template <int N> bool operator<(const Dual<N>& a, double b) { return a.v < b; }
// (sqrt s)' = s' / (2 sqrt s)
template <int N> Dual<N> sqrt(const Dual<N>& a) {
  Dual<N> r(std::sqrt(a.v));
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] / (2.0 * r.v);
  return r;
}

using D4 = Dual<4>;

}  // namespace

// ---------------------------------------------------------------------------------------
// C interface for the Python test harness (ctypes). Arrays are row-major [ny][nx] doubles;
// population arrays are [9][ny][nx] in the D2Q9 order above. Errors return a negative code.
// ---------------------------------------------------------------------------------------
extern "C" {

typedef Oracle<double> OracleD;

void* orc_create(const orc_params* p) {
  if (!p) return nullptr;
  Derived d;
  if (!derive(*p, &d)) return nullptr;
  OracleD* o = new (std::nothrow) OracleD();
  if (!o) return nullptr;
  o->p = *p;
  o->d = d;
  o->eps = p->eps;
  o->Dlat = d.Dlat;
  o->lambda = d.lambda;
  o->nx = p->nx;
  o->ny = p->ny;
  o->n = (size_t)p->nx * (size_t)p->ny;
  alloc(o);
  return o;
}

void orc_destroy(void* h) { delete static_cast<OracleD*>(h); }

// Derived lattice constants: Dphi, dt/tau0, D_lat, W0/dx, lambda, tau_f.
int orc_derived(void* h, double out[6]) {
  if (!h || !out) return -1;
  const Derived& d = static_cast<OracleD*>(h)->d;
  out[0] = d.Dphi; out[1] = d.dt_tau0; out[2] = d.Dlat;
  out[3] = d.Wlat; out[4] = d.lambda; out[5] = d.tau_f;
  return 0;
}

int orc_set_fields(void* h, const double* phi, const double* U, const double* rho,
                   const double* ux, const double* uy) {
  if (!h || !phi || !U) return -1;
  init_fields(static_cast<OracleD*>(h), phi, U, rho, ux, uy);
  return 0;
}

// Host threads of the node loops (1 by default); returns the number in use.
int orc_set_threads(int n) {
  omp_set_num_threads(n < 1 ? 1 : n);
  return omp_get_max_threads();
}

int orc_step(void* h, int64_t nsteps) {
  if (!h || nsteps < 0) return -1;
  OracleD* o = static_cast<OracleD*>(h);
  for (int64_t s = 0; s < nsteps; ++s) step_once(o);
  return 0;
}

int64_t orc_steps_done(void* h) { return h ? static_cast<OracleD*>(h)->steps : -1; }

int orc_get_field(void* h, int which, double* out) {
  if (!h || !out || which < 0 || which > 5) return -1;
  get_field(*static_cast<OracleD*>(h), which, out);
  return 0;
}

// lattice: 0 f, 1 g, 2 h. out/in: [9][ny][nx].
int orc_get_pops(void* h, int lattice, double* out) {
  if (!h || !out || lattice < 0 || lattice > 2) return -1;
  OracleD* o = static_cast<OracleD*>(h);
  if (lattice == 0 && !o->p.flow) return -1;
  const std::vector<double>* src = lattice == 0 ? o->f : lattice == 1 ? o->g : o->h;
  for (int a = 0; a < 9; ++a) std::memcpy(out + a * o->n, src[a].data(), o->n * sizeof(double));
  return 0;
}

int orc_set_pops(void* h, int lattice, const double* in) {
  if (!h || !in || lattice < 0 || lattice > 3) return -1;
  OracleD* o = static_cast<OracleD*>(h);
  if (lattice == 3) {  // phi history
    std::memcpy(o->phi_prev.data(), in, o->n * sizeof(double));
    return 0;
  }
  if (lattice == 0 && !o->p.flow) return -1;
  std::vector<double>* dst = lattice == 0 ? o->f : lattice == 1 ? o->g : o->h;
  for (int a = 0; a < 9; ++a) std::memcpy(dst[a].data(), in + a * o->n, o->n * sizeof(double));
  return 0;
}

// Test option: round the state (every population and the phi history) to float32 in place,
// the storage precision of an FP32 run, leaving the arithmetic of the next step in double.
int orc_round_f32(void* h) {
  if (!h) return -1;
  OracleD* o = static_cast<OracleD*>(h);
  std::vector<double>* lat[3] = {o->f, o->g, o->h};
  for (int L = 0; L < 3; ++L) {
    if (L == 0 && !o->p.flow) continue;
    for (int a = 0; a < 9; ++a) {
      double* v = lat[L][a].data();
#pragma omp parallel for schedule(static)
      for (long long i = 0; i < (long long)o->n; ++i) v[i] = (double)(float)v[i];
    }
  }
  double* ph = o->phi_prev.data();
#pragma omp parallel for schedule(static)
  for (long long i = 0; i < (long long)o->n; ++i) ph[i] = (double)(float)ph[i];
  return 0;
}

// Collision only, of the current state: lattice 0/1/2 -> f*, g*, h* as [9][ny][nx];
// lattice 3 -> a_s^2 as [ny][nx]. The state itself is not advanced.
int orc_post_collision(void* h, int lattice, double* out) {
  if (!h || !out || lattice < 0 || lattice > 3) return -1;
  OracleD* o = static_cast<OracleD*>(h);
  if (lattice == 0 && !o->p.flow) return -1;
  collide(o);
  if (lattice == 3) {
    std::memcpy(out, o->as2.data(), o->n * sizeof(double));
    return 0;
  }
  const std::vector<double>* src = lattice == 0 ? o->fs : lattice == 1 ? o->gs : o->hs;
  for (int a = 0; a < 9; ++a) std::memcpy(out + a * o->n, src[a].data(), o->n * sizeof(double));
  return 0;
}

// E4 isotropic gradient of a periodic field (Sec. 3.1.1), lattice units.
int orc_gradient_periodic(const double* phi, int nx, int ny, double* gx, double* gy) {
  if (!phi || !gx || !gy || nx < 1 || ny < 1) return -1;
  auto P = [&](int x, int y) {
    x = ((x % nx) + nx) % nx;
    y = ((y % ny) + ny) % ny;
    return phi[(size_t)y * nx + x];
  };
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x)
      grad_e4(P(x + 1, y), P(x - 1, y), P(x, y + 1), P(x, y - 1), P(x + 1, y + 1),
              P(x - 1, y + 1), P(x + 1, y - 1), P(x - 1, y - 1), &gx[(size_t)y * nx + x],
              &gy[(size_t)y * nx + x]);
  return 0;
}

// a_s and N (Sec. 2.1, R1) for one gradient vector: out = {a_s, N_x, N_y}.
int orc_anisotropy(double gx, double gy, double eps, double kappa_N, double out[3]) {
  if (!out) return -1;
  anisotropy(gx, gy, eps, kappa_N, 6, &out[0], &out[1], &out[2]);
  return 0;
}

// a_s and N for a given symmetry fold (4 or 6).
int orc_anisotropy_fold(double gx, double gy, double eps, double kappa_N, int fold,
                        double out[3]) {
  if (!out || (fold != 4 && fold != 6)) return -1;
  anisotropy(gx, gy, eps, kappa_N, fold, &out[0], &out[1], &out[2]);
  return 0;
}

// Gradient of a periodic field with a given stencil (2, 4, 6, 8), lattice units.
int orc_gradient_stencil(const double* phi, int nx, int ny, int stencil, double* gx,
                         double* gy) {
  if (!phi || !gx || !gy || nx < 1 || ny < 1) return -1;
  if (stencil != 2 && stencil != 4 && stencil != 6 && stencil != 8) return -1;
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      auto P = [&](int dx, int dy) {
        const int xx = (((x + dx) % nx) + nx) % nx, yy = (((y + dy) % ny) + ny) % ny;
        return phi[(size_t)yy * nx + xx];
      };
      gradient_stencil(stencil, P, &gx[(size_t)y * nx + x], &gy[(size_t)y * nx + x]);
    }
  return 0;
}

// Exact derivatives of the linear functional L = sum_x (wphi(x) phi_T(x) + wU(x) U_T(x)) of
// the state after nsteps steps from the equilibrium state of the given moments (R13), with
// respect to four directions: 0 eps; 1 D (through D_lat = D dt/dx^2 and, when lambda is not
// given, through the beta = 0 lambda = tau0 D / (a2 W0^2) of Sec. 2.1); 2 lambda alone;
// 3 the initial moments along (dphi, dU, drho, dux, duy). rho, ux, uy and their directions
// may be null (fluid at rest). out = {L, dL/d0, dL/d1, dL/d2, dL/d3}.
// round_f32 != 0: after every step the values (not the derivatives) of the populations and
// of the phi history are rounded to float, so the derivatives are those along a trajectory
// stored in float32 -- the spread against round_f32 = 0 measures how strongly the gradient
// reacts to storage rounding.
// along (may be null): states to differentiate along, nsteps + 1 blocks (the initial state,
// then the state after every step), each holding the planes h0..h8, g0..g8, [f0..f8,] phi,
// phi history, [ny][nx] each. The values (not the derivatives) of the state are replaced by
// block s before step s + 1, and the collision of that step takes its phi values from the
// block's phi plane, so the derivatives are those of the step linearised at the given states.
int orc_grad_run(const orc_params* p, const double* phi, const double* U, const double* rho,
                 const double* ux, const double* uy, const double* dphi, const double* dU,
                 const double* drho, const double* dux, const double* duy, int64_t nsteps,
                 const double* wphi, const double* wU, int32_t round_f32, const double* along,
                 double out[5]) {
  if (!p || !phi || !U || !dphi || !dU || !wphi || !wU || !out || nsteps < 0) return -1;
  Derived d;
  if (!derive(*p, &d)) return -1;
  Oracle<D4> o;
  o.p = *p;
  o.d = d;
  o.nx = p->nx;
  o.ny = p->ny;
  o.n = (size_t)p->nx * (size_t)p->ny;
  o.eps = D4(p->eps);
  o.eps.d[0] = 1.0;
  o.Dlat = D4(d.Dlat);
  o.Dlat.d[1] = p->dt / (p->dx * p->dx);
  o.lambda = D4(d.lambda);
  o.lambda.d[2] = 1.0;
  if (!(p->lambda > 0)) o.lambda.d[1] = p->tau0 / (kA2 * p->W0 * p->W0);
  alloc(&o);
  auto seeded = [&](const double* v, const double* dv) {
    std::vector<D4> r;
    if (!v) return r;
    r.resize(o.n);
    for (size_t i = 0; i < o.n; ++i) {
      r[i] = D4(v[i]);
      r[i].d[3] = dv ? dv[i] : 0.0;
    }
    return r;
  };
  init_fields_t(&o, seeded(phi, dphi), seeded(U, dU), seeded(rho, drho), seeded(ux, dux),
                seeded(uy, duy));
  auto round_values = [](std::vector<D4>& v) {
    for (D4& x : v) x.v = (double)(float)x.v;
  };
  const size_t nplanes = (p->flow ? 27 : 18) + 2;
  auto force = [&](int64_t s) {  // values of block s; its phi plane for the next collision
    const double* b = along + (size_t)s * nplanes * o.n;
    auto put = [&](std::vector<D4>& v, const double* src) {
      for (size_t i = 0; i < o.n; ++i) v[i].v = src[i];
    };
    for (int a = 0; a < 9; ++a) {
      put(o.h[a], b + (size_t)a * o.n);
      put(o.g[a], b + (size_t)(9 + a) * o.n);
      if (o.p.flow) put(o.f[a], b + (size_t)(18 + a) * o.n);
    }
    put(o.phi_prev, b + (nplanes - 1) * o.n);
    o.phi_force = b + (nplanes - 2) * o.n;
  };
  if (along) force(0);
  for (int64_t s = 0; s < nsteps; ++s) {
    step_once(&o);
    if (along) force(s + 1);
    if (round_f32) {
      for (int a = 0; a < 9; ++a) {
        round_values(o.h[a]);
        round_values(o.g[a]);
        if (o.p.flow) round_values(o.f[a]);
      }
      round_values(o.phi_prev);
    }
  }
  o.phi_force = nullptr;
  D4 L(0.0);
  D4 v[9];
  for (size_t i = 0; i < o.n; ++i) {
    for (int a = 0; a < 9; ++a) v[a] = o.h[a][i];
    const D4 ph = sum9(v);
    for (int a = 0; a < 9; ++a) v[a] = o.g[a][i];
    const D4 Ui = sum9(v);
    L = L + (wphi[i] * ph + wU[i] * Ui);
  }
  out[0] = L.v;
  for (int k = 0; k < 4; ++k) out[1 + k] = L.d[k];
  return 0;
}

}  // extern "C"
