// plan.h -- the plan object behind ibm_plan and helpers shared by the
// host-side translation units of libibm.
#pragma once

#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/ibm.h"
#include "internal.h"

namespace ibm {

int set_error(int code, const char *fmt, ...);
int cuda_error(cudaError_t e, const char *what);

#define IBM_CUDA_TRY(call)                                    \
  do {                                                        \
    cudaError_t e__ = (call);                                 \
    if (e__ != cudaSuccess) return ::ibm::cuda_error(e__, #call); \
  } while (0)

}  // namespace ibm

struct ibm_plan_s {
  int nx, ny, nz, P;
  int bc;            // IBM_BC_PXZ_WALL_Y or IBM_BC_TRIPLY_PERIODIC
  double h[3];
  int precision;     // IBM_FP64 / IBM_FP32_REFINED
  int refine;        // refinement steps (FP32 path)
  int delta;         // IBM_DELTA_*
  int pencil_mode;   // 0 auto, 1 warp-parallel block solve, 2 tile sweep, 3 streaming sweep, 4 segmented sweep
  int use_plane = 1; // plane mode: 0 split x / z passes; 1 one CTA per plane; C >= 2 a cluster of C CTAs per plane;
                     // -1 (kPlaneDft) tensor-core DFT products (FP32, short planes)
  int use_plane_fields = 0; // plane mode of three-field solves
  int use_slab = 0;  // FP32 single-field solves through the fused slab path (slab.cu)
  size_t esz;        // element size: 4 or 8
  size_t npts;       // nx * ny * nz
  size_t nspec;      // ny * nz * P complex entries
  void *S;           // spectrum workspace
  void *Sx[2];       // spectra of fields 1 and 2 of a three-field solve (allocated on first use)
  void *work;        // real work field (residual / divergence)
  void *bsave;       // copy of an in-place right-hand side
  void *sub[4];      // substep fields du, dv, dw, phi (allocated on first substep)
  void *mkbuf;       // marker force scratch [n][3] when the caller passes none
  size_t mkcap;      // bytes of mkbuf
  int spread = 0;    // IBM_SPREAD_ATOMIC / IBM_SPREAD_GATHER / IBM_SPREAD_ATOMIC_DIRECT
  void *gbuf = nullptr;  // gather-spreading workspace (bins, sorted entries, stencil records)
  size_t gcap = 0;       // bytes of gbuf
  void *twx, *twz;   // twiddles W_N^m (plan precision)
  void *dftf = nullptr, *dfti = nullptr;  // tensor-core DFT matrix tables (FP32 plans with short planes)
  void *twy, *lamy;  // triply periodic branch: W_ny^m and lambda_y (plan precision)
  void *lamx, *lamz; // modified wavenumbers kx'^2 (P), kz'^2 (nz) (plan precision)
  double *dsc;       // device scalars: [0] removed mean, [1] it as a float pair, [4..7] residual
                     // sums, [8..9] divergence maxima
  int *derr;         // device error word (bounded waits that gave up)
  double *zbuf;      // [2 ny] FP64 zero-pencil right-hand side and solution
  double *hsc;       // pinned host mirror of dsc
  cudaEvent_t ev0, ev1;
  size_t bytes;      // device bytes held
  // per-kernel tracing (ibm_plan_profile)
  struct ProfRec { int kind, launches; cudaEvent_t a, b; };
  int prof_on;
  std::vector<ProfRec> prof;
  std::vector<cudaEvent_t> evpool;
};

namespace ibm {
// Brackets the launches of one kernel kind with events when tracing is on.
struct ProfScope {
  ibm_plan_s *p;
  int kind, launches;
  cudaStream_t st;
  cudaEvent_t a = nullptr;
  ProfScope(ibm_plan_s *plan, int k, cudaStream_t s, int n = 1);
  ~ProfScope();
};
}  // namespace ibm

namespace ibm {
// Per-kind device times of one call for ibm_info::phase_ms: turns tracing on
// for the call (if it was off) and, at read(), sums the call's own event
// pairs by kind and drops them again, leaving any trace the caller is
// collecting with ibm_plan_profile untouched.
// Inactive (no info requested) it changes nothing.
struct InfoTrace {
  ibm_plan_s *p;
  size_t mark;
  int was_on;
  bool active;
  InfoTrace(ibm_plan_s *plan, bool on) : p(plan), mark(plan->prof.size()), was_on(plan->prof_on), active(on) {
    if (active) p->prof_on = 1;
  }
  void read(double *phase_ms);  // after the stream has drained
  ~InfoTrace() {
    if (active) p->prof_on = was_on;
  }
};
// The plan's device error word, read through stream st (after the work it
// reports on, which st must follow) and cleared: IBM_ERR_TIMEOUT when a
// bounded wait gave up, IBM_ERR_ARG when markers were rejected by the wall
// rule (with their count), else IBM_OK.  Synchronises st.
int plan_status(ibm_plan_s *p, cudaStream_t st);
inline bool aligned_to(const void *p, size_t a) { return ((uintptr_t)p % a) == 0; }
TransformGeom geom_of(const ibm_plan_s *p);
// Solve A x = b with the plan's direct method (+ refinement for FP32).
//   kind 0: Poisson L x = b (mean-free);  kind 1: Helmholtz (I - c L) x = b.
// out may equal in.  addend (nullable) is added to the result: out = addend + x.
int plan_solve(ibm_plan_s *p, int kind, double c, int field_bc, const void *in, void *out, const void *addend,
               cudaStream_t st, ibm_info *info);
// nb <= 3 Helmholtz solves (I - c L) x_b = in_b of one grid in the same
// launches, field b with boundary kind field_bc[b]: out_b = addend_b + x_b
// (no refinement: the increment form keeps the FP32 error relative to the
// addend).  Allocates the extra spectra on first use.
int plan_solve_fields(ibm_plan_s *p, double c, int nb, const int *field_bc, const void *const *in, void *const *out,
                      const void *const *addend, cudaStream_t st);

// Whether a plan of this kind takes the fused slab path for its single-field
// solves by default (FP32, wall branch, supported shape; IBM_SLAB=0 turns it
// off).
bool default_use_slab(int precision, int bc, int nx, int ny, int nz);

// One validated RK stage without info (substep.cu), and the allocation of
// every buffer a stage with nmk markers uses, so that a stage can be captured
// into a CUDA graph (no allocation during capture).
int substep_checked(ibm_plan_s *p, ibm_state *st, int rk_stage, double dt, double nu, ibm_markers *mk,
                    cudaStream_t stream);
int prepare_substep(ibm_plan_s *p, int nmk);
// (alpha_n + beta_n) dt: how far stage n advances the state time.
double stage_time_advance(int rk_stage, double dt);

// Autotuner result for one shape (batch.cu).
struct TuneChoice {
  int pencil_mode, use_plane;
  double ms;
};
// Times the solve variants of plan p (cached per shape), applies the fastest.
int tune_plan(ibm_plan_s *p, TuneChoice *out);
}  // namespace ibm
