// Declarations of the gas-kinetic (GKS) path: face kernel (Sec. 2.2 with Appendix A) and
// the two-stage fourth-order (S2O4) stage kernels.
#pragma once

#include <cuda_runtime.h>

#include "ase_df_internal.cuh"

namespace asedf {

struct GksSweepArgs {
  const double* W;        // [C][ny][nx]
  const double* s_norm;   // sigma of the faces normal to the sweep
  const double* s_tan;    // sigma of the faces along the sweep lines (2D)
  double* F;              // face flux (value at t_n) of this direction
  double* Ft;             // its time derivative
  double* s_out;          // sigma_out of this direction
  const DevState* st;     // dt of the step when dt_fixed <= 0
  double dt_fixed;        // > 0: the step's dt
  double inv_dn, inv_dt;  // 1/h along the sweep and across it
  double c1, c2;          // tau_n = c1 dt + c2 |p_l - p_r| / (p_l + p_r) dt
  double tfrac = 0.0;     // the stage's time is st->t + tfrac dt (time-dependent ghosts)
};

struct GksCombineArgs {
  const double *Fx, *Fxt, *Fy, *Fyt;  // face fluxes and their time derivatives
  const double* Wn;       // W^n
  double* out;            // stage 0: L; 1: W*; 2: W^{n+1}
  double* Lt_out;         // stage 0: L_t (else unused)
  double *L0, *Lt0;       // stage 1 writes L(W^n), L_t(W^n); stage 2 reads them
  DevState* st;
  double inv_dx, inv_dy;
  double dt_fixed;        // > 0: this dt, else st->dt
  int stage;              // 0: residual only; 1, 2: S2O4 stages
};

cudaError_t launch_gks_sweep_r3(int dim, int dir, const GridInfo& g, const GksSweepArgs& a, const Tables& t,
                                const DTables& d, cudaStream_t s);
cudaError_t launch_gks_sweep_r5(int dim, int dir, const GridInfo& g, const GksSweepArgs& a, const Tables& t,
                                const DTables& d, cudaStream_t s);
cudaError_t launch_gks_sweep_r7(int dim, int dir, const GridInfo& g, const GksSweepArgs& a, const Tables& t,
                                const DTables& d, cudaStream_t s);
cudaError_t launch_gks_sweep_r9(int dim, int dir, const GridInfo& g, const GksSweepArgs& a, const Tables& t,
                                const DTables& d, cudaStream_t s);

cudaError_t launch_gks_combine(int dim, const GridInfo& g, const GksCombineArgs& a, cudaStream_t s);
// st->dt := dt_fixed if > 0, else cfl / max speed (from the preceding max-speed reduction,
// and the inflow speed), shortened to t_end; raises the DT flag if it is not positive.
cudaError_t launch_gks_dt(DevState* st, double dt_fixed, double cfl, double t_end, double inflow_speed,
                          cudaStream_t s);

}  // namespace asedf
