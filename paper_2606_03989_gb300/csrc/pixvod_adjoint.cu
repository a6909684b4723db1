// Adjoint kernels of the sweep (reverse-mode per pixel, see pv_adjoint.cuh),
// compiled on their own: their launchers are called from pixvod.cu.
#include "pv_adjoint.cuh"

namespace pv {

cudaError_t launch_adjoint_sweep(const AdjArgs& A, int blocks, cudaStream_t st) {
    k_adjoint_sweep<<<blocks, ad::ADJ_THREADS, 0, st>>>(A);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_seed(const AdjArgs& A, const double* grad_xi, const double* grad_invdepth, double* adj,
                                cudaStream_t st) {
    dim3 block(32, 4), grid((A.g.W + 31) / 32, (A.g.H + 3) / 4);
    k_adjoint_seed<<<grid, block, 0, st>>>(A, grad_xi, grad_invdepth, adj);
    return cudaGetLastError();
}

cudaError_t launch_sigma_grads(const double* dparam, double sigma_D, double sigma_N, double* out, cudaStream_t st) {
    k_sigma_grads<<<1, 1, 0, st>>>(dparam, sigma_D, sigma_N, out);
    return cudaGetLastError();
}

}  // namespace pv
