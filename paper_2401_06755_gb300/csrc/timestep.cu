// The segregated multiphase time step of Section 2.4 on the GPU, assembled from the library's
// own entry points: Stage 1 (hydrostatic + surface-tension pressure, Eq. ph_disc), Stage 2 (the
// momentum predictor, Eq. velocity-1, `momentum_iters` times), Stage 3 (`correction_iters`
// non-hydrostatic pressure corrections, Eqs. ph_disc2 and vel-cor) and Stage 4 (the
// volume-fraction update, Eq. transport-indicator-1).  Both pressure equations have the
// constant-coefficient operator and the same faces, so one plan serves them.
#include <cstring>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace nn4 {
namespace {

struct FlowImpl {
  nn4_grid vg, pg;
  nn4_flow_params fp;
  nn4_plan plan = nullptr;
  size_t f = 0;  // elements per field (pitch * ny * nz)
  double* ws = nullptr;
  // views into ws
  double *src[3], *uh[3], *uh2[3], *ut[3], *un[3], *ptot, *b, *dp, *mom_ws, *vof_ws, *Cn, *sC;
  double* mass = nullptr;
  unsigned long long* range = nullptr;
};

__global__ void k_add(const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ out, size_t n) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
    out[t] = a[t] + b[t];
}

__device__ __forceinline__ double unord(unsigned long long v) {
  const unsigned long long b = (v & 0x8000000000000000ull) ? (v & 0x7FFFFFFFFFFFFFFFull) : ~v;
  return __longlong_as_double((long long)b);
}

__global__ void k_range_init(unsigned long long* r) {
  r[0] = ~0ull;
  r[1] = 0ull;
}

}  // namespace

int launch_range(const nn4_grid* g, const double* C, unsigned long long* out, cudaStream_t s);

}  // namespace nn4

using namespace nn4;

struct nn4_flow_s {
  FlowImpl* impl;
};

extern "C" {

int nn4_flow_create(const nn4_grid* vg, const nn4_grid* pg, const nn4_flow_params* fp, const nn4_plan_opts* popts,
                    nn4_flow* out) {
  if (!out || !vg || !pg || !fp) return set_error(NN4_EINVAL, "NULL argument");
  *out = nullptr;
  for (int d = 0; d < 3; ++d)
    if (vg->n[d] != pg->n[d] || vg->h[d] != pg->h[d]) return set_error(NN4_EINVAL, "velocity and pressure grids differ");
  if (vg->pitch != pg->pitch) return set_error(NN4_EINVAL, "velocity and pressure pitches differ");
  if (fp->momentum_iters < 1 || fp->correction_iters < 1 || (fp->pressure_rtol <= 0 && fp->pressure_cycles < 1))
    return set_error(NN4_EINVAL, "bad iteration counts");
  FlowImpl* F = new FlowImpl();
  F->vg = *vg;
  F->pg = *pg;
  F->fp = *fp;
  int rc = nn4_plan_create(pg, nullptr, popts, &F->plan);
  if (rc) {
    delete F;
    return rc;
  }
  F->f = (size_t)vg->pitch * vg->n[1] * vg->n[2];
  const int nfields = 3 + 3 + 3 + 3 + 3 + 1 + 1 + 1 + 3 + 3 + 1 + 1;
  cudaError_t e = cudaMalloc(&F->ws, sizeof(double) * F->f * nfields);
  if (e != cudaSuccess) {
    nn4_plan_destroy(F->plan);
    delete F;
    return check_cuda(e, "flow workspace");
  }
  cudaMemset(F->ws, 0, sizeof(double) * F->f * nfields);
  double* p = F->ws;
  auto take = [&](int n) {
    double* q = p;
    p += F->f * n;
    return q;
  };
  for (int c = 0; c < 3; ++c) F->src[c] = take(1);
  for (int c = 0; c < 3; ++c) F->uh[c] = take(1);
  for (int c = 0; c < 3; ++c) F->uh2[c] = take(1);
  for (int c = 0; c < 3; ++c) F->ut[c] = take(1);
  for (int c = 0; c < 3; ++c) F->un[c] = take(1);
  F->ptot = take(1);
  F->b = take(1);
  F->dp = take(1);
  F->mom_ws = take(3);
  F->vof_ws = take(3);
  F->Cn = take(1);
  F->sC = take(1);
  if ((rc = check_cuda(cudaMalloc(&F->mass, sizeof(double)), "flow scalars")) ||
      (rc = check_cuda(cudaMalloc(&F->range, 2 * sizeof(unsigned long long)), "flow scalars"))) {
    cudaFree(F->ws);
    nn4_plan_destroy(F->plan);
    delete F;
    return rc;
  }
  nn4_flow h = new nn4_flow_s;
  h->impl = F;
  *out = h;
  return NN4_OK;
}

int nn4_flow_destroy(nn4_flow f) {
  if (!f) return NN4_OK;
  FlowImpl* F = f->impl;
  nn4_plan_destroy(F->plan);
  cudaFree(F->ws);
  cudaFree(F->mass);
  cudaFree(F->range);
  delete F;
  delete f;
  return NN4_OK;
}

int nn4_flow_step(nn4_flow f, double* C, double* u, double* v, double* w, double* p_hs, double* p_nh,
                  nn4_flow_stats* stats, void* stream) {
  if (!f || !C || !u || !v || !w || !p_hs || !p_nh) return set_error(NN4_EINVAL, "NULL argument");
  FlowImpl* F = f->impl;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t fb = sizeof(double) * F->f;
  const nn4_flow_params& fp = F->fp;
  const bool fixed = fp.pressure_rtol <= 0.0;
  const double rtol = fixed ? 0.0 : fp.pressure_rtol;
  const int iters = fixed ? fp.pressure_cycles : 1000;
  int rc;
  nn4_solve_info info{};
  // Stage 1: sources at level n and the hydrostatic + surface-tension pressure
  if ((rc = nn4_momentum_sources(&F->vg, &fp, C, F->src[0], F->src[1], F->src[2], nullptr, nullptr, s)) ||
      (rc = nn4_pressure_rhs_hs_ex(&F->pg, fp.compute, F->src[0], F->src[1], F->src[2], F->b, s)))
    return rc;
  rc = nn4_pressure_solve(F->plan, F->b, p_hs, rtol, iters, &info, s);
  if (rc && rc != NN4_ENOCONV) return rc;
  if (stats) {
    stats->hs_iters = info.iterations;
    stats->hs_rel = info.rel_res;
  }
  // Stage 2: predictor iterations from u^{n+1/2} = u^n (the iterations alternate between two
  // u^{n+1/2} buffers: the filters read the current one around every node)
  double* vel[3] = {u, v, w};
  for (int c = 0; c < 3; ++c)
    if ((rc = check_cuda(cudaMemcpyAsync(F->un[c], vel[c], fb, cudaMemcpyDeviceToDevice, s), "copy u"))) return rc;
  const int blocks = (int)std::min<size_t>((F->f + 255) / 256, 152 * 16);
  k_add<<<blocks, 256, 0, s>>>(p_hs, p_nh, F->ptot, F->f);
  if ((rc = check_cuda(cudaGetLastError(), "p total"))) return rc;
  const double* unc[3] = {F->un[0], F->un[1], F->un[2]};
  const double* srcc[3] = {F->src[0], F->src[1], F->src[2]};
  for (int it = 0; it < fp.momentum_iters; ++it) {
    double* const* cur = it == 0 ? F->un : (it % 2 ? F->uh : F->uh2);
    double* const* nxt = it % 2 ? F->uh2 : F->uh;
    const double* cc[3] = {cur[0], cur[1], cur[2]};
    const bool last = it + 1 == fp.momentum_iters;
    if ((rc = nn4_momentum_predict(&F->vg, &fp, C, unc, cc, F->ut, last ? nullptr : nxt, F->ptot, srcc, F->mom_ws, s)))
      return rc;
  }
  // Stage 3: non-hydrostatic pressure corrections on u~
  for (int it = 0; it < fp.correction_iters; ++it) {
    if ((rc = nn4_pressure_rhs_nh(&F->pg, &fp, C, F->ut[0], F->ut[1], F->ut[2], F->b, nullptr, s))) return rc;
    if ((rc = check_cuda(cudaMemsetAsync(F->dp, 0, fb, s), "zero dp"))) return rc;
    rc = nn4_pressure_solve(F->plan, F->b, F->dp, rtol, iters, &info, s);
    if (rc && rc != NN4_ENOCONV) return rc;
    if ((rc = nn4_velocity_correct(&F->vg, &fp, C, F->dp, F->ut[0], F->ut[1], F->ut[2], p_nh, s))) return rc;
  }
  if (stats) {
    stats->nh_iters = info.iterations;
    stats->nh_rel = info.rel_res;
  }
  // u^{n+1} = u~; Stage 4 with q^{n+1}
  for (int c = 0; c < 3; ++c)
    if ((rc = check_cuda(cudaMemcpyAsync(vel[c], F->ut[c], fb, cudaMemcpyDeviceToDevice, s), "copy u"))) return rc;
  nn4_vof_params vp;
  nn4_vof_params_default(&vp, fp.dt);
  vp.compute = fp.compute;
  if ((rc = nn4_vof_advect_residual(&F->vg, &vp, C, u, v, w, F->sC, F->Cn, F->vof_ws, s))) return rc;
  if ((rc = check_cuda(cudaMemcpyAsync(C, F->Cn, fb, cudaMemcpyDeviceToDevice, s), "copy C"))) return rc;
  if (stats) {
    k_range_init<<<1, 1, 0, s>>>(F->range);
    if ((rc = nn4_mass_sum(&F->vg, C, F->mass, s)) || (rc = launch_range(&F->vg, C, F->range, s))) return rc;
    unsigned long long rg[2];
    double mass;
    if ((rc = check_cuda(cudaMemcpyAsync(&mass, F->mass, sizeof(double), cudaMemcpyDeviceToHost, s), "mass")) ||
        (rc = check_cuda(cudaMemcpyAsync(rg, F->range, sizeof(rg), cudaMemcpyDeviceToHost, s), "range")) ||
        (rc = check_cuda(cudaStreamSynchronize(s), "sync")))
      return rc;
    auto un_ord = [](unsigned long long x) {
      const unsigned long long b = (x & 0x8000000000000000ull) ? (x & 0x7FFFFFFFFFFFFFFFull) : ~x;
      double d;
      std::memcpy(&d, &b, sizeof(d));
      return d;
    };
    stats->mass = mass;
    stats->c_min = un_ord(rg[0]);
    stats->c_max = un_ord(rg[1]);
  }
  return check_cuda(cudaStreamSynchronize(s), "flow step");
}

}  // extern "C"
