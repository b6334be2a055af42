// Restarted FOM-LR on A^2 (Algorithm 1 with Section 5's rational sign): device state and launchers
// (implemented in kernels_fom.cu).
#pragma once

#include "kernels.h"

namespace ovl {

constexpr int kFomMaxK = 64;   // longest cycle (Arnoldi steps before a restart)
constexpr int kFomBlock = 128; // threads per block of the Gram-Schmidt kernels
constexpr int kFomMaxE = 8;    // elements per thread of the Gram-Schmidt kernels, at most

struct FomDev {
  size_t n = 0;            // 12 V
  int nrhs = 0, kcap = 0;  // right-hand sides, cycle length k
  int nblk = 0;            // partial slots per rhs (>= blocks of a Gram-Schmidt launch)
  int pstride = 0;         // doubles per block partial: 2 (kcap + 1)
  void* V = nullptr;       // [kcap+1][nrhs][n] basis v_0..v_k (FP64 or FP32 complex, native layout)
  double2* H = nullptr;    // [nrhs][kcap][kcap+1]: column j holds h_{0..j+1, j}
  double2* c1 = nullptr;   // [nrhs][kcap+1] first Gram-Schmidt coefficients of the current step
  double2* c2 = nullptr;   // [nrhs][kcap+1] second (reorthogonalisation) coefficients
  double* part = nullptr;  // [nrhs][nblk][pstride] block partials
  double* scale = nullptr; // [nrhs] 1 / h_{j+1,j} of the last step, or 1 / |r| at a cycle start
  double* beta = nullptr;  // [nrhs] |r| at the start of the cycle
  int* status = nullptr;   // [nrhs] 0 running, 1 invariant subspace reached in this cycle, 2 done
  int* kdone = nullptr;    // [nrhs] Arnoldi steps completed in this cycle
};

int fom_partial_slots(size_t n);
// Gram-Schmidt pass 0 / 1 / 2 of step j (see kernels_fom.cu): the block partials, then their sums
// in block order. j = -1 with pass 2: |v_0| of a cycle start (beta, scale).
cudaError_t launch_fom_gs(const FomDev& f, bool f64, int j, int pass, cudaStream_t st);
// v_{j+1} *= scale (j = -1: v_0)
cudaError_t launch_fom_scale(const FomDev& f, bool f64, int j, cudaStream_t st);
// x_P, r = (I - P) b into v_0 (unnormalised), X = 0; with m > 0 the deflation dots first.
cudaError_t launch_fom_start(const Geom& g, bool f64, const FomDev& f, const double2* b, int m, const double2* R,
                             const double2* L, const double* lam_sign, double2* dots, double* dpart, unsigned* dcount,
                             double2* xp, double2* X, cudaStream_t st);
// v_0 = (I - P) v_k (unnormalised) for every rhs that is not done.
cudaError_t launch_fom_restart(const Geom& g, bool f64, const FomDev& f, int k, int m, const double2* R,
                               const double2* L, double* part, unsigned* count, double2* d, cudaStream_t st);
// X += sum_{i < kr} coef_i v_i.
cudaError_t launch_fom_combine(const FomDev& f, bool f64, const int* kr, const double2* coef, double2* X,
                               cudaStream_t st);

}  // namespace ovl
