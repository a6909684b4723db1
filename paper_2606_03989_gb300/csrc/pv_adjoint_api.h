// Host-side view of the adjoint kernels (defined in pixvod_adjoint.cu): the
// per-sweep argument block and the launchers.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include "pv_kernels.cuh"

namespace pv {
namespace ad {
constexpr int ADJ_THREADS = 32;  // threads per block of the adjoint kernel

// Per-thread reverse-mode tapes: node n of thread slot s is at n * n_slots + s.
struct TapeCtl {
    int2* par;      // the two parents of each node (-1: none)
    double2* w;     // d node / d parent
    double* adj;    // adjoints of the reverse pass
    int cap;        // nodes per thread
    int n_slots;    // threads of the launch
};
}  // namespace ad

constexpr unsigned FLAG_TAPE_FULL = 0x8u;  // a pixel's tape overflowed: its gradient is missing

// Arguments of the adjoint of one sweep. State buffers and input planes hold
// FP64 when state64 is set, FP32 otherwise. The adjoint states are FP64 for the
// tape kernel and in the state's precision for the hand-written one; the
// gradients of the inputs and factor weights are FP64.
struct AdjArgs {
    Geometry<double> g;
    int state64;
    double lam_D, inv_sigma_D, lam_N, lam_P, lam_Z, lam_R, beta, t_huber, d_prior;
    const void* state_in;          // S_{s-1} (tile-major)
    const void* state_out;         // S_s, for the check of the recomputed update
    const void* adj_out;           // adjoint of S_s (tile-major, 151 planes)
    void* adj_in;                  // adjoint of S_{s-1}, accumulated
    const unsigned char* br;       // the sweep's recorded decisions (BR_*, tile-major pixel index)
    const void* I_s;               // input planes (row-major, pitched)
    const void* I_t;
    const void* g_x;
    const void* g_y;
    const void* m_x;
    const void* m_y;
    double* dI_s;                  // W x H, accumulated over the sweeps
    double* dI_t;
    double* dparam;                // adjoints of lam_D, 1/sigma_D, lam_N
    unsigned long long* mismatch;  // largest |recomputed - stored| / max(1, |stored|), as bits
    unsigned* max_nodes;           // longest tape of a pixel
    unsigned* flags;
    ad::TapeCtl tape;
    // hand-written pass: scale[0] = E, the adjoint state holds values in units
    // of 2^E; scale[1] = max |adj_out| in those units (as written by
    // launch_adjoint_absmax); the pass reads adj_out times 2^-e with
    // e = ilogb(scale[1]), so its adj_in is in units of 2^(E + e)
    double* scale;
};

// adjoint of one sweep by the reverse-mode tape (FP64), `blocks` blocks of
// ADJ_THREADS threads striding over the pixels
cudaError_t launch_adjoint_sweep(const AdjArgs& A, int blocks, cudaStream_t st);
// adjoint of one sweep by the hand-written reverse pass, in the state's
// precision, as ADJOINT_HW_LAUNCHES launches: per pixel and direction (the
// damped identity messages and what their reverse needs, summed over the
// directions), per pixel (the update and the reverse pass of everything but the
// identity messages), per pixel and direction (the identity messages' reverse
// pass), per tile (the recompute check), per pixel (the pose); `scratch`
// (adjoint_scratch_bytes) carries values between them
constexpr int ADJOINT_HW_LAUNCHES = 5;
size_t adjoint_scratch_bytes(int n_tiles, int state64);
cudaError_t launch_adjoint_hw(const AdjArgs& A, int n_tiles, void* scratch, cudaStream_t st);
// adjoint of xi_est = mean mu[0:6] and of the inverse depth exp(-mu[6]) at the
// state A.state_out, written into adj (all other planes left as they are), FP64
// (adj64) or FP32
cudaError_t launch_adjoint_seed(const AdjArgs& A, const double* grad_xi, const double* grad_invdepth, void* adj,
                                int adj64, cudaStream_t st);
// scale[1] = max |a[i]| over n elements (finite values; scale[1] must be 0 before),
// and z[i] = 0 over the same n elements (the next pass's adj_in)
cudaError_t launch_adjoint_absmax(const void* a, void* z, size_t n, int adj64, double* scale, cudaStream_t st);
// scale[0] += ilogb(scale[1]): the units of the adjoint state after a hand-written
// pass; scale[1] = 0 again for the next pass's absmax
cudaError_t launch_adjoint_exponent(double* scale, cudaStream_t st);
// dL/d(sigma_D, sigma_N) from the adjoints of lam_D, 1/sigma_D and lam_N
cudaError_t launch_sigma_grads(const double* dparam, double sigma_D, double sigma_N, double* out, cudaStream_t st);

}  // namespace pv
