// Explicit multiphase terms in FP64: the compressive Petrov-Galerkin volume-fraction update of
// Section 2.3 (Eqs. Petrov-C, Petrov-Cs, a_psi, efficient-kabs, Sx-lin, negativek,
// normalisation, positivek, alpha_min_and_max, transport-indicator-1) and the lumped-mass total
// of the mass diagnostic.  These kernels are FP64-ALU bound (several hundred flops per node on a
// part with 1.2 FP64 TFLOP/s), so they are plain one-thread-per-node kernels that read
// neighbours through L1; every Q1 filter is applied sum-factorised with boundary-aware 1D
// element factors (natural truncation).
#include <mutex>
#include <string>

#include "common.cuh"
#include "internal.h"

namespace nn4 {

NN4_DEFINE_ERROR_ACCESSOR(flow_error_word)

namespace {

struct FlowGeom {
  int nx, ny, nz;
  long long pitch;
  double h[3];
};

__device__ __forceinline__ long long fo(const FlowGeom& g, int i, int j, int k) {
  return i + g.pitch * ((long long)j + (long long)g.ny * k);
}

// 1D assembled Q1 factors at node i (n nodes, spacing h) for offset d in {-1, 0, 1}:
// K stiffness, M mass, G first derivative (int N_i dN_j/dx), L lumped (diagonal of M's rows).
struct F1 {
  double K[3], M[3], G[3], GT[3];  // GT: the transpose of the first-derivative filter
};

__device__ __forceinline__ F1 factors(int i, int n, double h) {
  const double eL = i > 0 ? 1.0 : 0.0, eR = i < n - 1 ? 1.0 : 0.0;
  F1 f;
  f.K[0] = -eL / h;
  f.K[1] = (eL + eR) / h;
  f.K[2] = -eR / h;
  f.M[0] = eL * h / 6.0;
  f.M[1] = (eL + eR) * h / 3.0;
  f.M[2] = eR * h / 6.0;
  f.G[0] = -0.5 * eL;
  f.G[1] = 0.5 * (eL - eR);
  f.G[2] = 0.5 * eR;
  f.GT[0] = 0.5 * eL;  // G[i-1][i] = +1/2 when node i-1 exists
  f.GT[1] = 0.5 * (eL - eR);
  f.GT[2] = -0.5 * eR;  // G[i+1][i] = -1/2 when node i+1 exists
  return f;
}

__device__ __forceinline__ double lumped(int i, int n, double h) {
  return 0.5 * h * ((i > 0) + (i < n - 1));
}

// sum_{dx,dy,dz} ax[dx] ay[dy] az[dz] f(i+dx, j+dy, k+dz) over existing neighbours (the factors
// of missing neighbours are zero; their index is clamped to stay in bounds).
__device__ __forceinline__ double tp(const FlowGeom& g, const double* __restrict__ f, int i, int j, int k,
                                     const double* ax, const double* ay, const double* az) {
  double sz = 0.0;
#pragma unroll
  for (int dz = -1; dz <= 1; ++dz) {
    const int kk = min(max(k + dz, 0), g.nz - 1);
    double sy = 0.0;
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy) {
      const int jj = min(max(j + dy, 0), g.ny - 1);
      const double* row = f + g.pitch * ((long long)jj + (long long)g.ny * kk);
      const double sx = ax[0] * row[max(i - 1, 0)] + ax[1] * row[i] + ax[2] * row[min(i + 1, g.nx - 1)];
      sy += ay[dy + 1] * sx;
    }
    sz += az[dz + 1] * sy;
  }
  return sz;
}

// Same with the product field a*b formed on the fly.
__device__ __forceinline__ double tp2(const FlowGeom& g, const double* __restrict__ a, const double* __restrict__ b,
                                      int i, int j, int k, const double* ax, const double* ay, const double* az) {
  double sz = 0.0;
#pragma unroll
  for (int dz = -1; dz <= 1; ++dz) {
    const int kk = min(max(k + dz, 0), g.nz - 1);
    double sy = 0.0;
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy) {
      const int jj = min(max(j + dy, 0), g.ny - 1);
      const long long r = g.pitch * ((long long)jj + (long long)g.ny * kk);
      const int il = max(i - 1, 0), ir = min(i + 1, g.nx - 1);
      const double sx = ax[0] * a[r + il] * b[r + il] + ax[1] * a[r + i] * b[r + i] + ax[2] * a[r + ir] * b[r + ir];
      sy += ay[dy + 1] * sx;
    }
    sz += az[dz + 1] * sy;
  }
  return sz;
}

#define NN4_NODE(G)                                        \
  const int i = blockIdx.x * blockDim.x + threadIdx.x;     \
  const int j = blockIdx.y * blockDim.y + threadIdx.y;     \
  const int k = blockIdx.z;                                \
  if (i >= (G).nx || j >= (G).ny) return;                  \
  const long long o = fo(G, i, j, k);

// Step 1: raw first-derivative filters f(C; w_d) and the advective derivative u . grad C with
// the pointwise gradient m^-1 f(C; w_d).
__global__ void k_vof_grad(const FlowGeom g, const double* __restrict__ C, const double* __restrict__ u,
                           const double* __restrict__ v, const double* __restrict__ w, double* __restrict__ fx,
                           double* __restrict__ fy, double* __restrict__ fz, double* __restrict__ gadv) {
  NN4_NODE(g)
  const F1 X = factors(i, g.nx, g.h[0]), Y = factors(j, g.ny, g.h[1]), Z = factors(k, g.nz, g.h[2]);
  const double m = lumped(i, g.nx, g.h[0]) * lumped(j, g.ny, g.h[1]) * lumped(k, g.nz, g.h[2]);
  const double gx = tp(g, C, i, j, k, X.G, Y.M, Z.M);
  const double gy = tp(g, C, i, j, k, X.M, Y.G, Z.M);
  const double gz = tp(g, C, i, j, k, X.M, Y.M, Z.G);
  fx[o] = gx;
  fy[o] = gy;
  fz[o] = gz;
  gadv[o] = (u[o] * gx + v[o] * gy + w[o] * gz) / m;
}

__device__ __forceinline__ double detector(const double* __restrict__ C, long long o, long long stride, int idx,
                                           int n) {
  const double c0 = C[o];
  const double cm = idx > 0 ? C[o - stride] : c0;  // copy-halo at walls
  const double cp = idx < n - 1 ? C[o + stride] : c0;
  return (c0 - cm) * (cp - c0);
}

// Step 2: the directional diffusion coefficients k^x, k^y, k^z.
__global__ void k_vof_coef(const FlowGeom g, const nn4_vof_params p, const double* __restrict__ C,
                           const double* __restrict__ fx, const double* __restrict__ fy,
                           const double* __restrict__ fz, const double* __restrict__ gadv,
                           const double* __restrict__ u, const double* __restrict__ v,
                           const double* __restrict__ w, double* __restrict__ kx, double* __restrict__ ky,
                           double* __restrict__ kz) {
  NN4_NODE(g)
  const F1 X = factors(i, g.nx, g.h[0]), Y = factors(j, g.ny, g.h[1]), Z = factors(k, g.nz, g.h[2]);
  const double m = lumped(i, g.nx, g.h[0]) * lumped(j, g.ny, g.h[1]) * lumped(k, g.nz, g.h[2]);
  const double cx = fx[o] / m, cy = fy[o] / m, cz = fz[o] / m;
  // Eq. a_psi: alpha_a f(u . grad C; w_m / m - E)
  const double a_C = p.alpha_a * (tp(g, gadv, i, j, k, X.M, Y.M, Z.M) / m - gadv[o]);
  // Eq. efficient-kabs (general spacing)
  const double ax = fabs(cx), ay = fabs(cy), az = fabs(cz);
  const double sabs = ax + ay + az;
  const double alpha_kabs = 1.0 / (8.0 * (double)(1 << p.p));
  const double k_abs = alpha_kabs * fabs(a_C) * (g.h[0] * ax + g.h[1] * ay + g.h[2] * az) /
                       (p.eps_k + sabs * sabs / 3.0);
  // Eqs. negativek and normalisation
  const double gradsq = cx * cx + cy * cy + cz * cz;
  const double uu = u[o], vv = v[o], ww = w[o];
  const double proj = (uu * cx + vv * cy + ww * cz) / (p.eps_x + gradsq);
  const double us = fabs(cx * proj) + fabs(cy * proj) + fabs(cz * proj);
  const double k_neg = -p.beta * (uu * uu + vv * vv + ww * ww) / (p.eps_x + gradsq * us / 3.0);
  // detectors with the override, weights, positive / negative parts, clamp (Eq. alpha_min_and_max)
  const double c0 = C[o];
  const bool over = c0 > p.detect_hi || c0 < p.detect_lo;
  const double hmax = fmax(g.h[0], fmax(g.h[1], g.h[2])), hmin = fmin(g.h[0], fmin(g.h[1], g.h[2]));
  const double kmin = p.alpha_min * hmax * hmax / p.dt, kmax = p.alpha_max * hmin * hmin / p.dt;
  const long long sy = g.pitch, sz = g.pitch * (long long)g.ny;
  const double S[3] = {over ? -1.0 : detector(C, o, 1, i, g.nx), over ? -1.0 : detector(C, o, sy, j, g.ny),
                       over ? -1.0 : detector(C, o, sz, k, g.nz)};
  double kd[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const double wp = -fmax(-1.0, fmin(0.0, p.K_plus * S[d]));
    const double wm = fmin(1.0, fmax(0.0, p.K_minus * S[d]));
    const double kk = wp * (p.K_pos * k_abs) + wm * (k_neg / g.h[d]);
    kd[d] = fmax(-kmin, fmin(kmax, kk));
  }
  kx[o] = kd[0];
  ky[o] = kd[1];
  kz[o] = kd[2];
}

// Step 3: s_C of Eq. Petrov-Cs and the update of Eq. transport-indicator-1.
__global__ void k_vof_update(const FlowGeom g, const nn4_vof_params p, const double* __restrict__ C,
                             const double* __restrict__ fx, const double* __restrict__ fy,
                             const double* __restrict__ fz, const double* __restrict__ kx,
                             const double* __restrict__ ky, const double* __restrict__ kz,
                             const double* __restrict__ u, const double* __restrict__ v,
                             const double* __restrict__ w, double* __restrict__ sC, double* __restrict__ Cn) {
  NN4_NODE(g)
  const F1 X = factors(i, g.nx, g.h[0]), Y = factors(j, g.ny, g.h[1]), Z = factors(k, g.nz, g.h[2]);
  const double m = lumped(i, g.nx, g.h[0]) * lumped(j, g.ny, g.h[1]) * lumped(k, g.nz, g.h[2]);
  double s = u[o] * fx[o] + v[o] * fy[o] + w[o] * fz[o];
  const double c0 = C[o];
  const double* kf[3] = {kx, ky, kz};
  // directional second-derivative filters w_dd^PG = K(d) x M x M, each in Eq. k-Txx form
  const double* ax[3] = {X.K, X.M, X.M};
  const double* ay[3] = {Y.M, Y.K, Y.M};
  const double* az[3] = {Z.M, Z.M, Z.K};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const double kc = kf[d][o];
    const double DkC = tp2(g, kf[d], C, i, j, k, ax[d], ay[d], az[d]);
    const double DC = tp(g, C, i, j, k, ax[d], ay[d], az[d]);
    const double Dk = tp(g, kf[d], i, j, k, ax[d], ay[d], az[d]);
    s += 0.5 * (DkC + kc * DC - c0 * Dk);
  }
  sC[o] = s;
  if (Cn) Cn[o] = c0 - p.dt * s / m;
}

// Lumped-mass total: sum_i m_i C_i in FP64 (one atomic per block).
__global__ void k_mass(const FlowGeom g, const double* __restrict__ C, double* out) {
  __shared__ double red[32];
  double s = 0.0;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i < g.nx && j < g.ny)
    s = lumped(i, g.nx, g.h[0]) * lumped(j, g.ny, g.h[1]) * lumped(k, g.nz, g.h[2]) * C[fo(g, i, j, k)];
  block_sum_atomic(s, out, red);
}


// ---------------------------------------------------------------- Navier-Stokes terms
__device__ __forceinline__ bool wall(const FlowGeom& g, int i, int j, int k, const int* dir) {
  return (dir[0] && i == 0) || (dir[1] && i == g.nx - 1) || (dir[2] && j == 0) || (dir[3] && j == g.ny - 1) ||
         (dir[4] && k == 0) || (dir[5] && k == g.nz - 1);
}

struct Faces {
  int d[6];
};

// Surface tension, step 1: the pointwise gradient of C and the normals n = grad C / (eps_t + |grad C|).
__global__ void k_st_normals(const FlowGeom g, const double* __restrict__ C, double eps_t, double* __restrict__ cd0,
                             double* __restrict__ cd1, double* __restrict__ cd2, double* __restrict__ n0,
                             double* __restrict__ n1, double* __restrict__ n2) {
  NN4_NODE(g)
  const F1 X = factors(i, g.nx, g.h[0]), Y = factors(j, g.ny, g.h[1]), Z = factors(k, g.nz, g.h[2]);
  const double m = lumped(i, g.nx, g.h[0]) * lumped(j, g.ny, g.h[1]) * lumped(k, g.nz, g.h[2]);
  const double gx = tp(g, C, i, j, k, X.G, Y.M, Z.M) / m;
  const double gy = tp(g, C, i, j, k, X.M, Y.G, Z.M) / m;
  const double gz = tp(g, C, i, j, k, X.M, Y.M, Z.G) / m;
  const double inv = 1.0 / (eps_t + sqrt(gx * gx + gy * gy + gz * gz));
  cd0[o] = gx;
  cd1[o] = gy;
  cd2[o] = gz;
  n0[o] = gx * inv;
  n1[o] = gy * inv;
  n2[o] = gz * inv;
}

// Surface tension, step 2: kappa = m^-1 sum_d f(n_d; w_d); s_d = sigma kappa C_d, and the total
// source s_z -= g rho (buoyancy) when `buoy` is set.
__global__ void k_st_source(const FlowGeom g, const double* __restrict__ C, const double* __restrict__ n0,
                            const double* __restrict__ n1, const double* __restrict__ n2, double* cd0, double* cd1,
                            double* cd2, double sigma, double gz_rho, double rho_l, double rho_g,
                            double* __restrict__ kappa) {
  NN4_NODE(g)
  const F1 X = factors(i, g.nx, g.h[0]), Y = factors(j, g.ny, g.h[1]), Z = factors(k, g.nz, g.h[2]);
  const double m = lumped(i, g.nx, g.h[0]) * lumped(j, g.ny, g.h[1]) * lumped(k, g.nz, g.h[2]);
  const double kap = (tp(g, n0, i, j, k, X.G, Y.M, Z.M) + tp(g, n1, i, j, k, X.M, Y.G, Z.M) +
                      tp(g, n2, i, j, k, X.M, Y.M, Z.G)) / m;
  if (kappa) kappa[o] = kap;
  const double rho = rho_l * C[o] + rho_g * (1.0 - C[o]);
  // in place: the gradient fields become the source fields (each node only reads its own values)
  cd0[o] = sigma * kap * cd0[o];
  cd1[o] = sigma * kap * cd1[o];
  cd2[o] = sigma * kap * cd2[o] - gz_rho * rho;
}

// Stage-1 right-hand side: b = sum_d G_d^T s_d (0 on Dirichlet nodes of the pressure grid).
__global__ void k_rhs_hs(const FlowGeom g, const double* __restrict__ s0, const double* __restrict__ s1,
                         const double* __restrict__ s2, const Faces pf, double* __restrict__ b) {
  NN4_NODE(g)
  if (wall(g, i, j, k, pf.d)) {
    b[o] = 0.0;
    return;
  }
  const F1 X = factors(i, g.nx, g.h[0]), Y = factors(j, g.ny, g.h[1]), Z = factors(k, g.nz, g.h[2]);
  b[o] = tp(g, s0, i, j, k, X.GT, Y.M, Z.M) + tp(g, s1, i, j, k, X.M, Y.GT, Z.M) + tp(g, s2, i, j, k, X.M, Y.M, Z.GT);
}

// Stage-3 right-hand side (Eq. ph_disc2): b = -(1/dt) sum_d [ f(rho u_d; w_d) - u_d f(rho; w_d) ]
// with rho = rho_l C + rho_g (1 - C) formed on the fly.
__global__ void k_rhs_nh(const FlowGeom g, const double* __restrict__ C, const double* __restrict__ u0,
                         const double* __restrict__ u1, const double* __restrict__ u2, double rho_l, double rho_g,
                         double dt, const Faces pf, double* __restrict__ b, double* __restrict__ rho_tmp) {
  NN4_NODE(g)
  if (wall(g, i, j, k, pf.d)) {
    b[o] = 0.0;
    return;
  }
  const F1 X = factors(i, g.nx, g.h[0]), Y = factors(j, g.ny, g.h[1]), Z = factors(k, g.nz, g.h[2]);
  const double* uu[3] = {u0, u1, u2};
  const double* ax[3] = {X.G, X.M, X.M};
  const double* ay[3] = {Y.M, Y.G, Y.M};
  const double* az[3] = {Z.M, Z.M, Z.G};
  double s = 0.0;
#pragma unroll
  for (int d = 0; d < 3; ++d)
    s += tp2(g, rho_tmp, uu[d], i, j, k, ax[d], ay[d], az[d]) - uu[d][o] * tp(g, rho_tmp, i, j, k, ax[d], ay[d], az[d]);
  b[o] = -s / dt;
}

__global__ void k_density(const FlowGeom g, const double* __restrict__ C, double rho_l, double rho_g,
                          double* __restrict__ rho) {
  NN4_NODE(g)
  rho[o] = rho_l * C[o] + rho_g * (1.0 - C[o]);
}

// Eq. vel-cor and the updates: u_d += -dt m^-1 f(dp; w_d) / rho (0 on velocity walls); p += dp.
__global__ void k_vel_correct(const FlowGeom g, const double* __restrict__ C, const double* __restrict__ dp,
                              double rho_l, double rho_g, double dt, const Faces vf, double* u0, double* u1,
                              double* u2, double* p) {
  NN4_NODE(g)
  const F1 X = factors(i, g.nx, g.h[0]), Y = factors(j, g.ny, g.h[1]), Z = factors(k, g.nz, g.h[2]);
  const double m = lumped(i, g.nx, g.h[0]) * lumped(j, g.ny, g.h[1]) * lumped(k, g.nz, g.h[2]);
  const double rho = rho_l * C[o] + rho_g * (1.0 - C[o]);
  if (!wall(g, i, j, k, vf.d)) {
    const double f = -dt / (m * rho);
    u0[o] += f * tp(g, dp, i, j, k, X.G, Y.M, Z.M);
    u1[o] += f * tp(g, dp, i, j, k, X.M, Y.G, Z.M);
    u2[o] += f * tp(g, dp, i, j, k, X.M, Y.M, Z.G);
  }
  if (p) p[o] += dp[o];
}

// Momentum, pass A for component psi: raw first-derivative filters and g = u^{n+1/2} . grad psi.
__global__ void k_mom_grad(const FlowGeom g, const double* __restrict__ psi, const double* __restrict__ uh0,
                           const double* __restrict__ uh1, const double* __restrict__ uh2, double* __restrict__ r0,
                           double* __restrict__ r1, double* __restrict__ r2, double* __restrict__ gp) {
  NN4_NODE(g)
  const F1 X = factors(i, g.nx, g.h[0]), Y = factors(j, g.ny, g.h[1]), Z = factors(k, g.nz, g.h[2]);
  const double m = lumped(i, g.nx, g.h[0]) * lumped(j, g.ny, g.h[1]) * lumped(k, g.nz, g.h[2]);
  const double a = tp(g, psi, i, j, k, X.G, Y.M, Z.M), b = tp(g, psi, i, j, k, X.M, Y.G, Z.M),
               c = tp(g, psi, i, j, k, X.M, Y.M, Z.G);
  r0[o] = a;
  r1[o] = b;
  r2[o] = c;
  gp[o] = (uh0[o] * a + uh1[o] * b + uh2[o] * c) / m;
}

// Momentum, pass B: k_psi = rho min(k_max, k_abs, k_square) + mu (Eqs. a_psi, efficient-kabs,
// h_Psi, k-square, max-k, k_Psi-n).
__global__ void k_mom_coef(const FlowGeom g, const nn4_flow_params fp, const double* __restrict__ C,
                           const double* __restrict__ r0, const double* __restrict__ r1,
                           const double* __restrict__ r2, const double* __restrict__ gp,
                           const double* __restrict__ uh0, const double* __restrict__ uh1,
                           const double* __restrict__ uh2, double* __restrict__ kpsi) {
  NN4_NODE(g)
  const F1 X = factors(i, g.nx, g.h[0]), Y = factors(j, g.ny, g.h[1]), Z = factors(k, g.nz, g.h[2]);
  const double m = lumped(i, g.nx, g.h[0]) * lumped(j, g.ny, g.h[1]) * lumped(k, g.nz, g.h[2]);
  const double px = r0[o] / m, py = r1[o] / m, pz = r2[o] / m;
  const double a = fp.alpha_a * (tp(g, gp, i, j, k, X.M, Y.M, Z.M) / m - gp[o]);
  const double ax = fabs(px), ay = fabs(py), az = fabs(pz), sab = ax + ay + az;
  const double hsum = g.h[0] * ax + g.h[1] * ay + g.h[2] * az;
  const double p2 = (double)(1 << fp.p);
  const double k_abs = (1.0 / (8.0 * p2)) * fabs(a) * hsum / (fp.eps_k + sab * sab / 3.0);
  const double h_psi = hsum / (fp.eps_k + sab);
  const double u0 = uh0[o], u1 = uh1[o], u2 = uh2[o];
  const double k_sq = (8.0 / p2) * a * a * h_psi /
                      (fp.eps_k + (fabs(u0 * px) + fabs(u1 * py) + fabs(u2 * pz)) * (px * px + py * py + pz * pz) / 3.0);
  const double kmax = g.h[0] * fabs(u0) + g.h[1] * fabs(u1) + g.h[2] * fabs(u2);
  const double c = C[o];
  const double rho = fp.rho_l * c + fp.rho_g * (1.0 - c), mu = fp.mu_l * c + fp.mu_g * (1.0 - c);
  kpsi[o] = rho * fmin(kmax, fmin(k_abs, k_sq)) + mu;
}

// Momentum, pass C: s~ (Eq. Petrov-u/v/w) and the predictor (Eq. velocity-1, sigma = 0):
// psi~ = psi^n - dt s~ / (m rho) (0 on walls); psi^{n+1/2}_new = (psi^n + psi~) / 2.
__global__ void k_mom_update(const FlowGeom g, const nn4_flow_params fp, int comp, const double* __restrict__ C,
                             const double* __restrict__ psi_n, const double* __restrict__ psi_h,
                             const double* __restrict__ r0, const double* __restrict__ r1,
                             const double* __restrict__ r2, const double* __restrict__ kpsi,
                             const double* __restrict__ uh0, const double* __restrict__ uh1,
                             const double* __restrict__ uh2, const double* __restrict__ ptot,
                             const double* __restrict__ src, const Faces vf, double* __restrict__ psi_t,
                             double* __restrict__ psi_half_out) {
  NN4_NODE(g)
  const F1 X = factors(i, g.nx, g.h[0]), Y = factors(j, g.ny, g.h[1]), Z = factors(k, g.nz, g.h[2]);
  const double m = lumped(i, g.nx, g.h[0]) * lumped(j, g.ny, g.h[1]) * lumped(k, g.nz, g.h[2]);
  const double c = C[o];
  const double rho = fp.rho_l * c + fp.rho_g * (1.0 - c);
  double s = rho * (uh0[o] * r0[o] + uh1[o] * r1[o] + uh2[o] * r2[o]);
  // viscous + PG term f^lap(psi, k; w_lap), the isotropic Q1 Laplacian = sum_d K_d x M x M
  const double kc = kpsi[o], pc = psi_h[o];
  const double* ax[3] = {X.K, X.M, X.M};
  const double* ay[3] = {Y.M, Y.K, Y.M};
  const double* az[3] = {Z.M, Z.M, Z.K};
  double Lkp = 0.0, Lp = 0.0, Lk = 0.0;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    Lkp += tp2(g, kpsi, psi_h, i, j, k, ax[d], ay[d], az[d]);
    Lp += tp(g, psi_h, i, j, k, ax[d], ay[d], az[d]);
    Lk += tp(g, kpsi, i, j, k, ax[d], ay[d], az[d]);
  }
  s += 0.5 * (Lkp + kc * Lp - pc * Lk);
  // pressure gradient f(p; w_comp) and consistent-mass source f(s_comp; w_m)
  const double* gx = comp == 0 ? X.G : X.M;
  const double* gy = comp == 1 ? Y.G : Y.M;
  const double* gz = comp == 2 ? Z.G : Z.M;
  s += tp(g, ptot, i, j, k, gx, gy, gz);
  s -= tp(g, src, i, j, k, X.M, Y.M, Z.M);
  const double pn = psi_n[o];
  const double pt = wall(g, i, j, k, vf.d) ? 0.0 : pn - fp.dt * s / (m * rho);
  psi_t[o] = pt;
  if (psi_half_out) psi_half_out[o] = 0.5 * (pn + pt);
}

__global__ void k_half(const FlowGeom g, const double* __restrict__ a, const double* __restrict__ b,
                       double* __restrict__ out) {
  NN4_NODE(g)
  out[o] = 0.5 * (a[o] + b[o]);
}

// min / max of a field (order-preserving integer image of doubles; out[0] = min, out[1] = max)
__device__ __forceinline__ unsigned long long ord(double v) {
  const unsigned long long b = __double_as_longlong(v);
  return (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);
}
__global__ void k_range(const FlowGeom g, const double* __restrict__ C, unsigned long long* out) {
  NN4_NODE(g)
  const unsigned long long v = ord(C[o]);
  atomicMin(&out[0], v);
  atomicMax(&out[1], v);
}

FlowGeom flow_geom(const nn4_grid* g) {
  FlowGeom f;
  f.nx = g->n[0];
  f.ny = g->n[1];
  f.nz = g->n[2];
  f.pitch = g->pitch;
  for (int d = 0; d < 3; ++d) f.h[d] = g->h[d];
  return f;
}

}  // namespace

int validate_grid(const nn4_grid* g, nn4_dtype dt, int min_n);
int validate_ptr(const void* p, const char* name);

}  // namespace nn4

using namespace nn4;

extern "C" {

void nn4_vof_params_default(nn4_vof_params* p, double dt) {
  if (!p) return;
  p->dt = dt;
  p->alpha_a = 2.0;
  p->eps_k = 1e-7;
  p->K_plus = 300.0;
  p->K_minus = 300.0;
  p->beta = 0.1;
  p->eps_x = 1e-4;
  p->K_pos = 3.0;
  p->alpha_min = 1e-4;
  p->alpha_max = 0.05;
  p->detect_hi = 0.95;
  p->detect_lo = 0.05;
  p->p = 1;
}

int64_t nn4_vof_workspace_bytes(const nn4_grid* g) {
  if (!g || g->pitch <= 0) return -1;
  return 7LL * g->pitch * g->n[1] * g->n[2] * (int64_t)sizeof(double);
}

int nn4_vof_advect_residual(const nn4_grid* g, const nn4_vof_params* p, const double* C, const double* u,
                            const double* v, const double* w, double* s_C, double* C_next, void* workspace,
                            void* stream) {
  int rc;
  if ((rc = validate_grid(g, NN4_F64, 2)) || (rc = validate_ptr(C, "C")) || (rc = validate_ptr(u, "u")) ||
      (rc = validate_ptr(v, "v")) || (rc = validate_ptr(w, "w")) || (rc = validate_ptr(s_C, "s_C")) ||
      (rc = validate_ptr(workspace, "workspace")))
    return rc;
  if (!p) return set_error(NN4_EINVAL, "params is NULL");
  if (!(p->dt > 0.0) || p->p < 1 || p->p > 3) return set_error(NN4_EINVAL, "bad VOF parameters");
  if (C_next && (rc = validate_ptr(C_next, "C_next"))) return rc;
  if (s_C == C || C_next == C) return set_error(NN4_EINVAL, "outputs must not alias C");
  const FlowGeom fg = flow_geom(g);
  const size_t f = (size_t)g->pitch * g->n[1] * g->n[2];
  double* ws = static_cast<double*>(workspace);
  double *fx = ws, *fy = ws + f, *fz = ws + 2 * f, *ga = ws + 3 * f, *kx = ws + 4 * f, *ky = ws + 5 * f,
         *kz = ws + 6 * f;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  dim3 blk(32, 4), grd((fg.nx + 31) / 32, (fg.ny + 3) / 4, fg.nz);
  k_vof_grad<<<grd, blk, 0, s>>>(fg, C, u, v, w, fx, fy, fz, ga);
  k_vof_coef<<<grd, blk, 0, s>>>(fg, *p, C, fx, fy, fz, ga, u, v, w, kx, ky, kz);
  k_vof_update<<<grd, blk, 0, s>>>(fg, *p, C, fx, fy, fz, kx, ky, kz, u, v, w, s_C, C_next);
  return check_cuda(cudaGetLastError(), "VOF kernels");
}

// ---------------------------------------------------------------- allocation-free variant
// The same three kernels with their scratch in a fixed device array instead of a caller buffer.
// Every GPU that loads the library holds this array (44 MiB) until the process exits.
constexpr long long kVofStaticFieldElems = 786432;  // max pitch * ny * nz per scratch field
static __device__ __align__(256) double g_vof_scratch[7 * kVofStaticFieldElems];

namespace {
std::mutex g_vof_scratch_mu;
double* g_vof_scratch_ptr[128] = {nullptr};  // device address of g_vof_scratch, per device ordinal
}  // namespace

int nn4_vof_advect_residual_static(const nn4_grid* g, const nn4_vof_params* p, const double* C, const double* u,
                                   const double* v, const double* w, double* s_C, double* C_next, void* stream) {
  int rc;
  if ((rc = validate_grid(g, NN4_F64, 2)) || (rc = validate_ptr(C, "C")) || (rc = validate_ptr(u, "u")) ||
      (rc = validate_ptr(v, "v")) || (rc = validate_ptr(w, "w")) || (rc = validate_ptr(s_C, "s_C")))
    return rc;
  if (!p) return set_error(NN4_EINVAL, "params is NULL");
  if (!(p->dt > 0.0) || p->p < 1 || p->p > 3) return set_error(NN4_EINVAL, "bad VOF parameters");
  if (C_next && (rc = validate_ptr(C_next, "C_next"))) return rc;
  if (s_C == C || C_next == C) return set_error(NN4_EINVAL, "outputs must not alias C");
  const long long f = (long long)g->pitch * g->n[1] * g->n[2];
  if (f > kVofStaticFieldElems)
    return set_error(NN4_EINVAL, "grid too large for the static scratch: pitch * ny * nz = " + std::to_string(f) +
                                     " > " + std::to_string(kVofStaticFieldElems));
  // set-up once per device, with that device current: the host-side name of the array is not a
  // device address, so take the address from the runtime
  int dev = 0;
  if ((rc = check_cuda(cudaGetDevice(&dev), "cudaGetDevice"))) return rc;
  if (dev < 0 || dev >= 128) return set_error(NN4_EUNSUPPORTED, "device ordinal out of range");
  double* ws = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_vof_scratch_mu);
    if (!g_vof_scratch_ptr[dev]) {
      void* ptr = nullptr;
      if ((rc = check_cuda(cudaGetSymbolAddress(&ptr, g_vof_scratch), "cudaGetSymbolAddress(scratch)"))) return rc;
      g_vof_scratch_ptr[dev] = static_cast<double*>(ptr);
    }
    ws = g_vof_scratch_ptr[dev];
  }
  // every scratch element the kernels read is written earlier in the same call (all nodes of the
  // seven fields), so nothing needs clearing between calls
  const FlowGeom fg = flow_geom(g);
  double *fx = ws, *fy = ws + f, *fz = ws + 2 * f, *ga = ws + 3 * f, *kx = ws + 4 * f, *ky = ws + 5 * f,
         *kz = ws + 6 * f;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  dim3 blk(32, 4), grd((fg.nx + 31) / 32, (fg.ny + 3) / 4, fg.nz);
  k_vof_grad<<<grd, blk, 0, s>>>(fg, C, u, v, w, fx, fy, fz, ga);
  k_vof_coef<<<grd, blk, 0, s>>>(fg, *p, C, fx, fy, fz, ga, u, v, w, kx, ky, kz);
  k_vof_update<<<grd, blk, 0, s>>>(fg, *p, C, fx, fy, fz, kx, ky, kz, u, v, w, s_C, C_next);
  return check_cuda(cudaGetLastError(), "VOF kernels (static scratch)");
}

void nn4_flow_params_default(nn4_flow_params* p, double dt) {
  if (!p) return;
  p->dt = dt;
  p->rho_l = 1000.0;
  p->rho_g = 1.0;
  p->mu_l = 1e-3;
  p->mu_g = 1.8e-5;
  p->sigma_t = 0.07;
  p->g = 9.81;
  p->alpha_a = 2.0;
  p->eps_k = 1e-7;
  p->p = 1;
  p->momentum_iters = 2;
  p->correction_iters = 2;
  p->pressure_cycles = 20;
  p->pressure_rtol = 0.0;
}

static Faces faces_of(const nn4_grid* g) {
  Faces f;
  for (int i = 0; i < 6; ++i) f.d[i] = g->bc[i] == NN4_BC_DIRICHLET ? 1 : 0;
  return f;
}

static int check_fp(const nn4_flow_params* fp) {
  if (!fp) return set_error(NN4_EINVAL, "flow params NULL");
  if (!(fp->dt > 0.0) || !(fp->rho_l > 0.0) || !(fp->rho_g > 0.0) || fp->p < 1 || fp->p > 3)
    return set_error(NN4_EINVAL, "bad flow parameters");
  return NN4_OK;
}

int nn4_momentum_sources(const nn4_grid* g, const nn4_flow_params* fp, const double* C, double* s0, double* s1,
                         double* s2, double* kappa, double* workspace, void* stream) {
  int rc;
  if ((rc = validate_grid(g, NN4_F64, 2)) || (rc = check_fp(fp)) || (rc = validate_ptr(C, "C")) ||
      (rc = validate_ptr(s0, "s0")) || (rc = validate_ptr(s1, "s1")) || (rc = validate_ptr(s2, "s2")) ||
      (rc = validate_ptr(workspace, "workspace")))
    return rc;
  const FlowGeom fg = flow_geom(g);
  const size_t f = (size_t)g->pitch * g->n[1] * g->n[2];
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  dim3 blk(32, 4), grd((fg.nx + 31) / 32, (fg.ny + 3) / 4, fg.nz);
  const double hmin = fmin(g->h[0], fmin(g->h[1], g->h[2]));
  k_st_normals<<<grd, blk, 0, st>>>(fg, C, 1e-7 / hmin, s0, s1, s2, workspace, workspace + f, workspace + 2 * f);
  k_st_source<<<grd, blk, 0, st>>>(fg, C, workspace, workspace + f, workspace + 2 * f, s0, s1, s2, fp->sigma_t, fp->g,
                                   fp->rho_l, fp->rho_g, kappa);
  return check_cuda(cudaGetLastError(), "momentum sources");
}

int nn4_pressure_rhs_hs(const nn4_grid* g, const double* s0, const double* s1, const double* s2, double* b,
                        void* stream) {
  int rc;
  if ((rc = validate_grid(g, NN4_F64, 2)) || (rc = validate_ptr(s0, "s0")) || (rc = validate_ptr(s1, "s1")) ||
      (rc = validate_ptr(s2, "s2")) || (rc = validate_ptr(b, "b")))
    return rc;
  const FlowGeom fg = flow_geom(g);
  dim3 blk(32, 4), grd((fg.nx + 31) / 32, (fg.ny + 3) / 4, fg.nz);
  k_rhs_hs<<<grd, blk, 0, static_cast<cudaStream_t>(stream)>>>(fg, s0, s1, s2, faces_of(g), b);
  return check_cuda(cudaGetLastError(), "stage-1 rhs");
}

int nn4_pressure_rhs_nh(const nn4_grid* g, const nn4_flow_params* fp, const double* C, const double* u,
                        const double* v, const double* w, double* b, double* rho_ws, void* stream) {
  int rc;
  if ((rc = validate_grid(g, NN4_F64, 2)) || (rc = check_fp(fp)) || (rc = validate_ptr(C, "C")) ||
      (rc = validate_ptr(u, "u")) || (rc = validate_ptr(v, "v")) || (rc = validate_ptr(w, "w")) ||
      (rc = validate_ptr(b, "b")) || (rc = validate_ptr(rho_ws, "rho_ws")))
    return rc;
  const FlowGeom fg = flow_geom(g);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  dim3 blk(32, 4), grd((fg.nx + 31) / 32, (fg.ny + 3) / 4, fg.nz);
  k_density<<<grd, blk, 0, st>>>(fg, C, fp->rho_l, fp->rho_g, rho_ws);
  k_rhs_nh<<<grd, blk, 0, st>>>(fg, C, u, v, w, fp->rho_l, fp->rho_g, fp->dt, faces_of(g), b, rho_ws);
  return check_cuda(cudaGetLastError(), "stage-3 rhs");
}

int nn4_velocity_correct(const nn4_grid* g, const nn4_flow_params* fp, const double* C, const double* dp, double* u,
                         double* v, double* w, double* p_nh, void* stream) {
  int rc;
  if ((rc = validate_grid(g, NN4_F64, 2)) || (rc = check_fp(fp)) || (rc = validate_ptr(C, "C")) ||
      (rc = validate_ptr(dp, "dp")) || (rc = validate_ptr(u, "u")) || (rc = validate_ptr(v, "v")) ||
      (rc = validate_ptr(w, "w")))
    return rc;
  const FlowGeom fg = flow_geom(g);
  dim3 blk(32, 4), grd((fg.nx + 31) / 32, (fg.ny + 3) / 4, fg.nz);
  k_vel_correct<<<grd, blk, 0, static_cast<cudaStream_t>(stream)>>>(fg, C, dp, fp->rho_l, fp->rho_g, fp->dt,
                                                                    faces_of(g), u, v, w, p_nh);
  return check_cuda(cudaGetLastError(), "velocity correction");
}

int nn4_momentum_predict(const nn4_grid* g, const nn4_flow_params* fp, const double* C, const double* const* un,
                         double* const* uh, double* const* ut, const double* p, const double* const* src,
                         double* workspace, void* stream) {
  int rc;
  if ((rc = validate_grid(g, NN4_F64, 2)) || (rc = check_fp(fp)) || (rc = validate_ptr(C, "C")) ||
      (rc = validate_ptr(p, "p")) || (rc = validate_ptr(workspace, "workspace")))
    return rc;
  if (!un || !uh || !ut || !src) return set_error(NN4_EINVAL, "NULL component array");
  for (int c = 0; c < 3; ++c)
    if ((rc = validate_ptr(un[c], "un")) || (rc = validate_ptr(uh[c], "uh")) || (rc = validate_ptr(ut[c], "ut")) ||
        (rc = validate_ptr(src[c], "s")))
      return rc;
  const FlowGeom fg = flow_geom(g);
  const size_t f = (size_t)g->pitch * g->n[1] * g->n[2];
  double *r0 = workspace, *r1 = workspace + f, *r2 = workspace + 2 * f, *gp = workspace + 3 * f, *kp = workspace + 4 * f;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  dim3 blk(32, 4), grd((fg.nx + 31) / 32, (fg.ny + 3) / 4, fg.nz);
  const Faces vf = faces_of(g);
  // u^{n+1/2} is read by all three components: update it only after all three u~ are known
  for (int c = 0; c < 3; ++c) {
    k_mom_grad<<<grd, blk, 0, st>>>(fg, uh[c], uh[0], uh[1], uh[2], r0, r1, r2, gp);
    k_mom_coef<<<grd, blk, 0, st>>>(fg, *fp, C, r0, r1, r2, gp, uh[0], uh[1], uh[2], kp);
    k_mom_update<<<grd, blk, 0, st>>>(fg, *fp, c, C, un[c], uh[c], r0, r1, r2, kp, uh[0], uh[1], uh[2], p, src[c], vf,
                                      ut[c], nullptr);
  }
  for (int c = 0; c < 3; ++c) k_half<<<grd, blk, 0, st>>>(fg, un[c], ut[c], uh[c]);
  return check_cuda(cudaGetLastError(), "momentum predictor");
}

}  // extern "C"

namespace nn4 {
int launch_range(const nn4_grid* g, const double* C, unsigned long long* out, cudaStream_t s) {
  const FlowGeom fg = flow_geom(g);
  dim3 blk(32, 4), grd((fg.nx + 31) / 32, (fg.ny + 3) / 4, fg.nz);
  k_range<<<grd, blk, 0, s>>>(fg, C, out);
  return check_cuda(cudaGetLastError(), "range");
}
}  // namespace nn4

extern "C" {

int nn4_mass_sum(const nn4_grid* g, const double* C, double* out, void* stream) {
  int rc;
  if ((rc = validate_grid(g, NN4_F64, 2)) || (rc = validate_ptr(C, "C"))) return rc;
  if (!out) return set_error(NN4_EINVAL, "out is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if ((rc = check_cuda(cudaMemsetAsync(out, 0, sizeof(double), s), "zero mass"))) return rc;
  const FlowGeom fg = flow_geom(g);
  dim3 blk(32, 4), grd((fg.nx + 31) / 32, (fg.ny + 3) / 4, fg.nz);
  k_mass<<<grd, blk, 0, s>>>(fg, C, out);
  return check_cuda(cudaGetLastError(), "mass sum");
}

}  // extern "C"
