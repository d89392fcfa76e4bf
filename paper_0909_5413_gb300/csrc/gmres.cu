// gmres.cu -- restarted GMRES(m) with right preconditioning for one problem
// (Sec. 2.2: GMRES with the RASM preconditioner; Sec. 3.1: relative tolerance
// 1e-13). A single problem is solved as a batch of one by the batched solver
// (gmres_batch.cu): the same per-chunk Gram-Schmidt passes, fixed-order
// reductions and device-side Givens, with the Arnoldi cycle replayed as a CUDA
// graph and one host read of the residual per cycle (restart or refinement
// step) instead of one per Arnoldi step.
//
//   FP64 form: V (m+1) x N in FP64, classical Gram-Schmidt applied twice;
//   mixed form: the cycle on FP32 vectors with the FP32 matvec and FP32
//   subdomain inverses (FP64-class dot products, FP64 Hessenberg and Givens),
//   one inner cycle per FP64 iterative-refinement step on the true FP64
//   residual.
#include "common.cuh"

namespace rbf {

rbf_status gmres_solve(rbf_ctx* ctx, const double* f, double* w, const rbf_solve_params* p, rbf_solve_info* info,
                       cudaStream_t st)
{
    return gmres_solve_batch(ctx, f, w, p, info, st);
}

}  // namespace rbf
