// FP64 vector kernels (reductions, MINRES/CG steps, line-search updates).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

namespace tmop {

constexpr int kMaxRedBlocks = 1024;

// Device scalar slots of the Krylov state (an array of doubles).
enum {
  KS_ALPHA = 0, KS_BETA, KS_BETA_NEXT2, KS_BETA_NEXT, KS_BETA1, KS_ETA, KS_C_OLD, KS_S_OLD, KS_C, KS_S,
  KS_R1, KS_R2, KS_INV_RHO, KS_PHI, KS_INV_BETA_NEXT, KS_RESID,
  KS_RR, KS_A, KS_B, KS_BREAKDOWN,
  KS_COUNT
};

int red_grid(size_t n);
int dot(const double* a, const double* b, size_t n, double* part, double* out, cudaStream_t s);
int energy_final(const double* pf, const double* pm, int np, double* outF, double* outMin, cudaStream_t s);
int step(const double* x, const double* p, double alpha, double* y, size_t n, cudaStream_t s);
int minres_init(const double* b, double* v, double* vprev, double* w, double* wprev, double* sol, double* st,
                double* part, size_t n, cudaStream_t s);
int minres_after_hv(double* v, double* vprev, double* Av, double* w, double* wprev, double* sol, double* st,
                    double* part, size_t n, cudaStream_t s);
int cg_init(const double* b, double* r, double* d, double* sol, double* st, double* part, size_t n,
            cudaStream_t s);
int cg_after_hv(double* sol, double* r, double* d, const double* Hd, double* st, double* part, size_t n,
                cudaStream_t s);

}  // namespace tmop
