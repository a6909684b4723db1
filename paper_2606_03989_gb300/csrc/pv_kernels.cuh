// PixVOD sweep kernels (templated on the arithmetic type).
//
// State: structure-of-arrays planes stored tile-major: the image is cut into
// 32 x 4-pixel tiles and each tile keeps all its planes contiguously
// (plane p of the tile's pixel `lane` at tile_base + p * 128 + lane), so plane
// offsets are compile-time constants and a tile's message planes are one
// contiguous block for a bulk copy. Two buffers are ping-ponged: a sweep reads
// one and writes every plane of the other. Planes:
//   0..6     mu (xi_0..xi_5, log-depth d)
//   7..27    M_p: pose information of the belief without the photometric factor
//            (pose prior plus the four identity messages), 6x6 packed lower
//   28..33   u: photometric part of the depth-marginalised pose information,
//            P = M_p + u u^T
//   34       s: belief information of the depth with the pose marginalised
//   35+27k   identity-factor message into the pixel from slot k: Lambda (21
//            packed lower) then eta (6); slots 0 left, 1 right, 2 up, 3 down
//   143+2k   normal-integration message from slot k: Lambda, eta
//
// After every sweep the stored beliefs are projected to the new linearisation
// point, where their eta is zero; the variable-to-factor message of pixel j
// towards a pairwise factor f is then belief minus that factor's message, and
// its marginal on the factor's dims is (P_j - Lambda_{f->j}, -eta_{f->j}) for an
// identity factor and (s_j - n_{f->j}, -e_{f->j}) for a normal factor, because
// each of those messages lives on one block (pose or depth) only. P_j is kept
// as M_p + u u^T because a single pixel's rank-one photometric information can
// exceed its other pose information by more than float32 resolves.
#pragma once

#include "pv_branch.h"
#include "pv_math.cuh"

namespace pv {

constexpr int N_PLANES = 151;
constexpr int PL_MU = 0;
constexpr int PL_MP = 7;
constexpr int PL_U = 28;
constexpr int PL_S = 34;
constexpr int PL_ID = 35;
constexpr int ID_STRIDE = 27;
constexpr int PL_NM = 143;
constexpr int N_INPUT_PLANES = 6;  // I_s, I_t, g_x, g_y, m_x, m_y (row-major, pitched)
constexpr int MSG_PLANES = PL_NM - PL_ID;  // 108: the identity-message planes 35..142
constexpr int TILE_W = 32;
constexpr int TILE_H = 4;
constexpr int TILE_PX = TILE_W * TILE_H;
constexpr int TILE_WORDS = N_PLANES * TILE_PX;

constexpr unsigned FLAG_NONPOS_PIVOT = 0x1u;
constexpr unsigned FLAG_NONFINITE = 0x2u;
constexpr unsigned FLAG_TIMEOUT = 0x4u;
constexpr unsigned FLAG_BOUNDS = 0x10u;  // checked builds: an index left its buffer (access skipped)

// Checked builds (PIXVOD_CHECKED): every computed index of the sweep (neighbour
// state, input planes, bilinear taps, shared-memory message slots) is tested
// against its buffer; a violation sets FLAG_BOUNDS in *flags and yields
// `fallback` (0) so the access is skipped. Plain builds compile the index as is.
#ifdef PIXVOD_CHECKED
#define PV_IDX(idx, limit, flags) (((size_t)(idx) < (size_t)(limit)) ? (size_t)(idx) : ((flags) |= FLAG_BOUNDS, (size_t)0))
#else
#define PV_IDX(idx, limit, flags) ((size_t)(idx))
#endif

// Device-resident per-handle scalars (doubles, fixed layout; the checkpoint
// format copies the first 40).
struct Scalars {
    double xi_est[6];
    double T_kf[16];   // T_kf<-world
    double T_cur[16];  // T_cam<-world of the last frame
    double d_prior;    // log-depth prior mean of the current keyframe segment
    double d_mean;     // mean log-depth after the last reduction
    unsigned flags;
    unsigned counter;  // last-block ticket of the reduction
    double pad[6];
};

template <typename T>
struct Geometry {
    int W, H, pitch;   // input planes: row-major with `pitch` elements per row
    size_t plane;      // elements per input plane
    int tiles_x;       // state: tiles per tile row
    T fx, fy, cx, cy, ifx, ify;
};

// element offset of pixel (u, v) in a tile-major state buffer (plane 0)
__host__ __device__ __forceinline__ size_t state_index(int u, int v, int tiles_x) {
    return (size_t)((v / TILE_H) * tiles_x + (u / TILE_W)) * TILE_WORDS + (v % TILE_H) * TILE_W + (u % TILE_W);
}

template <typename T>
struct Factors {
    T lam_D, inv_sigma_D, t_huber, lam_P, lam_R, lam_N, lam_Z, beta;
};

template <typename T>
struct SweepArgs {
    Geometry<T> g;
    Factors<T> f;
    const T* __restrict__ in;
    T* __restrict__ out;
    const T* __restrict__ I_s;
    const T* __restrict__ I_t;
    const T* __restrict__ g_x;
    const T* __restrict__ g_y;
    const T* __restrict__ m_x;
    const T* __restrict__ m_y;
    Scalars* sc;
    // when set, each pixel's discrete decisions of this sweep (BR_* bits) are
    // written here (tile-major pixel index), for the adjoint
    unsigned char* br;
};


// ---------------------------------------------------------------------------
// a0: frame ingest
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void normal_slopes(const float* __restrict__ n, int u, int v, const Geometry<T>& g,
                                              T* ax, T* ay) {
    T nx = T(n[0]), ny = T(n[1]), nz = T(n[2]);
    T nr = nx * (T(u) - g.cx) / g.fx + ny * (T(v) - g.cy) / g.fy + nz;
    bool ok = v_abs(nr) >= T(1e-3);
    *ax = ok ? nx / (g.fx * nr) : T(0);
    *ay = ok ? ny / (g.fy * nr) : T(0);
}

// Keyframe: source intensities and the normal-integration edge measurements of
// Eq. 6 (m_x between (u, v) and (u+1, v), m_y between (u, v) and (u, v+1)).
template <typename T>
__device__ __forceinline__ void ingest_keyframe_px(const Geometry<T>& g, const float* __restrict__ frame,
                                                   const float* __restrict__ normals, T* I_s, T* m_x, T* m_y,
                                                   int u, int v) {
    size_t i = (size_t)v * g.pitch + u;
    size_t f = (size_t)v * g.W + u;
    I_s[i] = T(frame[f]);
    T ax, ay;
    normal_slopes(normals + 3 * f, u, v, g, &ax, &ay);
    T mx = T(0), my = T(0);
    if (u + 1 < g.W) {
        T bx, by;
        normal_slopes(normals + 3 * (f + 1), u + 1, v, g, &bx, &by);
        mx = T(0.5) * (ax + bx);
    }
    if (v + 1 < g.H) {
        T bx, by;
        normal_slopes(normals + 3 * (f + g.W), u, v + 1, g, &bx, &by);
        my = T(0.5) * (ay + by);
    }
    m_x[i] = mx;
    m_y[i] = my;
}

template <typename T>
__global__ void k_ingest_keyframe(Geometry<T> g, const float* __restrict__ frame,
                                  const float* __restrict__ normals, T* I_s, T* m_x, T* m_y) {
    int u = blockIdx.x * blockDim.x + threadIdx.x;
    int v = blockIdx.y * blockDim.y + threadIdx.y;
    if (u >= g.W || v >= g.H) return;
    ingest_keyframe_px(g, frame, normals, I_s, m_x, m_y, u, v);
}

// Target: intensities and central-difference gradients (replicated borders).
template <typename T>
__device__ __forceinline__ void ingest_target_px(const Geometry<T>& g, const float* __restrict__ frame, T* I_t,
                                                 T* g_x, T* g_y, int u, int v) {
    size_t i = (size_t)v * g.pitch + u;
    const float* row = frame + (size_t)v * g.W;
    int ul = u > 0 ? u - 1 : 0, ur = u + 1 < g.W ? u + 1 : g.W - 1;
    int vu = v > 0 ? v - 1 : 0, vd = v + 1 < g.H ? v + 1 : g.H - 1;
    I_t[i] = T(row[u]);
    g_x[i] = T(0.5) * (T(row[ur]) - T(row[ul]));
    g_y[i] = T(0.5) * (T(frame[(size_t)vd * g.W + u]) - T(frame[(size_t)vu * g.W + u]));
}

template <typename T>
__global__ void k_ingest_target(Geometry<T> g, const float* __restrict__ frame, T* I_t, T* g_x, T* g_y) {
    int u = blockIdx.x * blockDim.x + threadIdx.x;
    int v = blockIdx.y * blockDim.y + threadIdx.y;
    if (u >= g.W || v >= g.H) return;
    ingest_target_px(g, frame, I_t, g_x, g_y, u, v);
}

// Keyframe reset: identity pose, log-depth at the segment's prior mean, no
// messages, belief equal to the priors (M_p = lam_P I, u = 0, s = lam_Z).
template <typename T>
__device__ __forceinline__ void reset_px(const Geometry<T>& g, const Factors<T>& f, T* state, const Scalars* sc,
                                         int u, int v) {
    T* st = state + state_index(u, v, g.tiles_x);
    T d0 = T(sc->d_prior);
    for (int p = 0; p < N_PLANES; ++p) st[p * TILE_PX] = T(0);
    st[6 * TILE_PX] = d0;
#pragma unroll
    for (int k = 0; k < 6; ++k) st[(PL_MP + pidx(k, k)) * TILE_PX] = f.lam_P;
    st[PL_S * TILE_PX] = f.lam_Z;
}

// Checked builds: the lanes of ragged tiles that lie outside the image hold NaN
// in every plane, so that any computation reading them shows as FLAG_NONFINITE.
template <typename T>
__global__ void k_poison_outside(Geometry<T> g, int n_tiles, T* state) {
    const int tile = blockIdx.x, lane = threadIdx.x;
    const int u = (tile % g.tiles_x) * TILE_W + lane % TILE_W;
    const int v = (tile / g.tiles_x) * TILE_H + lane / TILE_W;
    if (tile >= n_tiles || (u < g.W && v < g.H)) return;
    T* st = state + (size_t)tile * TILE_WORDS + lane;
    for (int p = 0; p < N_PLANES; ++p) st[p * TILE_PX] = T(NAN);
}

template <typename T>
__global__ void k_reset(Geometry<T> g, Factors<T> f, T* state, const Scalars* sc) {
    int u = blockIdx.x * blockDim.x + threadIdx.x;
    int v = blockIdx.y * blockDim.y + threadIdx.y;
    if (u >= g.W || v >= g.H) return;
    reset_px(g, f, state, sc, u, v);
}

// ---------------------------------------------------------------------------
// a1-a4: one synchronous sweep (v1: one thread per pixel, global loads)
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T bilinear(const T* __restrict__ img, int pitch, int x0, int y0, int x1, int y1,
                                      T ax, T ay) {
    T a = img[(size_t)y0 * pitch + x0], b = img[(size_t)y0 * pitch + x1];
    T c = img[(size_t)y1 * pitch + x0], d = img[(size_t)y1 * pitch + x1];
    return (T(1) - ay) * ((T(1) - ax) * a + ax * b) + ay * ((T(1) - ax) * c + ax * d);
}

// ---------------------------------------------------------------------------
// bulk (TMA) copies global -> shared with an mbarrier, in inline PTX
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// dst, src and bytes must be multiples of 16 bytes
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}
// bounded wait for phase `parity`; false if it did not complete
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity) {
    for (int it = 0; it < (1 << 22); ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// Loads of the swept state bypass L1 (ld.global.cg): the persistent batched
// kernel reads, after a grid barrier, data other SMs wrote in the same launch,
// and an SM's L1 is not kept coherent with those writes.
template <typename T>
__device__ __forceinline__ T ld_state(const T* p) {
    return __ldcg(p);
}

// Thread block of the sweep kernel: one state tile (32 x 4 pixels), one thread
// per pixel; 4 blocks per SM (55 KB of shared memory and at most 128 registers
// each). Each thread keeps its four damped identity messages in shared memory
// until the belief solve has given tau; their eta is then projected in place and
// the tile's 108 message planes leave with one bulk copy. The identity-message
// loop is not unrolled; the normal messages are computed in a loop of their own
// after it and stay in registers.
constexpr int SWEEP_BX = TILE_W;
constexpr int SWEEP_BY = TILE_H;
constexpr int SWEEP_THREADS = TILE_PX;

template <typename T>
constexpr size_t sweep_smem_bytes() {
    return sizeof(T) * MSG_PLANES * TILE_PX;
}

// The calling thread's pixel of the sweep over tile (tx, ty): everything but the
// store of the identity messages, which are left, projected, in `msg`. False if
// the tile's bulk copy never arrived (FLAG_TIMEOUT is set).
template <typename T>
__device__ __forceinline__ bool sweep_pixel(const SweepArgs<T>& a, int tx, int ty, T* msg, uint64_t* bar,
                                            unsigned parity) {
    const int tid = threadIdx.y * SWEEP_BX + threadIdx.x;
    const int u = tx * SWEEP_BX + threadIdx.x;
    const int v = ty * SWEEP_BY + threadIdx.y;
    const Geometry<T>& g = a.g;
    const Factors<T>& F = a.f;
    const size_t tile = (size_t)ty * g.tiles_x + tx;
    if (u >= g.W || v >= g.H) return true;
    unsigned flags = 0;
    const size_t n_state = (size_t)g.tiles_x * ((g.H + TILE_H - 1) / TILE_H) * TILE_WORDS;
    const size_t n_plane = g.plane;
    (void)n_state;
    (void)n_plane;
    const int i = (int)PV_IDX(v * g.pitch + u, n_plane, flags);
    const T* __restrict__ Si = a.in + PV_IDX(tile * TILE_WORDS + tid, n_state, flags);   // this pixel, plane 0
    T* __restrict__ Di = a.out + PV_IDX(tile * TILE_WORDS + tid, n_state, flags);

    T xi[6], d;
#pragma unroll
    for (int k = 0; k < 6; ++k) xi[k] = ld_state(Si + k * TILE_PX);
    d = ld_state(Si + 6 * TILE_PX);
    T R[9], t[3];
    se3_exp(xi, R, t);

    // The belief has the exact structure
    //   Lambda_b = blockdiag(M_p, m_d) + alpha J J^T,  eta_b = eta_o - alpha r J
    // (identity messages and the pose prior act on the pose block, normal messages
    // and the depth prior on the depth, the photometric factor is rank one), so it
    // is kept in that form: M_p (packed), m_d, alpha, J, r and eta_o (in eb).
    T eb[7];
#pragma unroll
    for (int q = 0; q < 7; ++q) eb[q] = T(0);
    // --- priors (Eq. 4 with identity Jacobian; log-depth prior) ---
    T Mp[21];
#pragma unroll
    for (int q = 0; q < 21; ++q) Mp[q] = T(0);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        Mp[pidx(k, k)] = F.lam_P;
        eb[k] -= F.lam_P * xi[k];
    }
    T md = F.lam_Z;
    eb[6] -= F.lam_Z * (d - T(a.sc->d_prior));

    // --- a2/a3: pairwise messages from the four neighbours ---
    if (!mbar_wait_bounded(bar, parity)) {
        // the tile's messages never arrived: flag it, wait once more, leave the tile
        atomicOr(&a.sc->flags, FLAG_TIMEOUT);
        mbar_wait_bounded(bar, parity);
        return false;
    }
    const T beta = F.beta, omb = T(1) - F.beta;
#pragma unroll 1
    for (int k = 0; k < 4; ++k) {
        T* mb = msg + PV_IDX((k * ID_STRIDE) * TILE_PX + tid, (MSG_PLANES - ID_STRIDE + 1) * TILE_PX, flags);  // slot k
        const int un = u + (k == 0 ? -1 : (k == 1 ? 1 : 0));
        const int vn = v + (k == 2 ? -1 : (k == 3 ? 1 : 0));
        const bool has = un >= 0 && un < g.W && vn >= 0 && vn < g.H;
        if (!has) {
#pragma unroll
            for (int q = 0; q < ID_STRIDE; ++q) mb[q * TILE_PX] = T(0);
            continue;
        }
        const int ko = k ^ 1;
        const T* Sj = a.in + PV_IDX(state_index(un, vn, g.tiles_x), n_state, flags);
        // variable-to-factor marginal of j: V = W + u u^T with W = M_p,j - Lambda_{f->j}
        // (pose prior plus j's three other identity messages) and u = u_j, and
        // eta_v = -eta_{f->j}. All of j's loads are issued here, ahead of the Exp/Log
        // chain of the residual, so that their latency overlaps it.
        const T* mj = Sj + (PL_ID + ID_STRIDE * ko) * TILE_PX;
        T W[21], C[21], z[6], gv[6];
        T uz = T(0), ur = T(0), uh = T(0);
        T uj[6], xj[6];
#pragma unroll
        for (int q = 0; q < 6; ++q) xj[q] = ld_state(Sj + q * TILE_PX);
#pragma unroll
        for (int q = 0; q < 21; ++q) W[q] = ld_state(Sj + (PL_MP + q) * TILE_PX) - ld_state(mj + q * TILE_PX);
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            uj[q] = ld_state(Sj + (PL_U + q) * TILE_PX);
            gv[q] = -ld_state(mj + (21 + q) * TILE_PX);
        }
        // identity factor (Eq. 5): r = Log(Exp(xi_j)^-1 Exp(xi_i)), J_i = I, J_j = -I
        T rb[6];
        {
            T Rj[9], tj[3], Rr[9], tr[3];
            se3_exp(xj, Rj, tj);
            se3_invmul(Rj, tj, R, t, Rr, tr);
            se3_log(Rr, tr, rb);
        }
        {
#pragma unroll
            for (int q = 0; q < 21; ++q) C[q] = W[q];
            // g0 = eta_v - W r
#pragma unroll
            for (int q = 0; q < 6; ++q) {
                T wr = T(0);
#pragma unroll
                for (int c = 0; c < 6; ++c) wr += W[pidx(q, c)] * rb[c];
                gv[q] -= wr;
            }
            // A = W + lam_R I is well conditioned (its eigenvalues are at least lam_R);
            // the rank-one u u^T, which can be far larger, stays out of the factorisation
#pragma unroll
            for (int q = 0; q < 6; ++q) C[pidx(q, q)] += F.lam_R;
            T idg0[6];
            if (!chol_packed<6>(C, idg0)) flags |= FLAG_NONPOS_PIVOT;
#pragma unroll
            for (int q = 0; q < 6; ++q) z[q] = uj[q];
            fwd_solve<6>(C, idg0, z);
            bwd_solve<6>(C, idg0, z);   // z = A^-1 u
            fwd_solve<6>(C, idg0, gv);
            bwd_solve<6>(C, idg0, gv);  // h = A^-1 g0
#pragma unroll
            for (int q = 0; q < 6; ++q) {
                uz += uj[q] * z[q];
                ur += uj[q] * rb[q];
                uh += uj[q] * gv[q];
                C[pidx(q, q)] = idg0[q];  // keep 1/L_qq on the diagonal (the solves below read it there)
            }
        }
        const T iuz = v_div(T(1), T(1) + uz);
        const T crank = F.lam_R * F.lam_R * iuz;
        // with C = A + u u^T (Sherman-Morrison):
        // eta_msg = lam_R C^-1 (eta_v - V r) = lam_R (h - z (u^T r + u^T h) / (1 + u^T z))
        const T ecoef = (ur + uh) * iuz;
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            T e = omb * (F.lam_R * (gv[q] - ecoef * z[q])) + beta * mb[(21 + q) * TILE_PX];
            eb[q] += e;
            mb[(21 + q) * TILE_PX] = e;
        }
        // Lambda_msg = lam_R C^-1 V = lam_R A^-1 W + lam_R^2 / (1 + u^T z) z z^T, the first
        // term (equal to W - W A^-1 W) one column at a time, rows c..5 of column c; this
        // product form has no cancellation for W << lam_R (~ W) or W >> lam_R (~ lam_R I)
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            T x[6];
#pragma unroll
            for (int r = 0; r < 6; ++r) x[r] = W[pidx(r, c)];
            fwd_solve_id<6>(C, x);
            bwd_solve_id<6>(C, x);
#pragma unroll
            for (int r = c; r < 6; ++r) {
                T l = omb * (F.lam_R * x[r] + crank * z[r] * z[c]) + beta * mb[pidx(r, c) * TILE_PX];
                Mp[pidx(r, c)] += l;
                mb[pidx(r, c) * TILE_PX] = l;
            }
        }

    }

    // normal-integration factors (Eq. 6): r_i = d_i - d_j + sg m
    T nl[4], ne[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        nl[k] = T(0);
        ne[k] = T(0);
        const int un = u + (k == 0 ? -1 : (k == 1 ? 1 : 0));
        const int vn = v + (k == 2 ? -1 : (k == 3 ? 1 : 0));
        if (!(un >= 0 && un < g.W && vn >= 0 && vn < g.H)) continue;
        const int ko = k ^ 1;
        const T* Sj = a.in + PV_IDX(state_index(un, vn, g.tiles_x), n_state, flags);
        T dj = ld_state(Sj + 6 * TILE_PX);
        T sv = ld_state(Sj + PL_S * TILE_PX) - ld_state(Sj + (PL_NM + 2 * ko) * TILE_PX);
        T evn = -ld_state(Sj + (PL_NM + 2 * ko + 1) * TILE_PX);
        T m = k == 0 ? a.m_x[PV_IDX(i - 1, n_plane, flags)]
                     : (k == 1 ? a.m_x[i] : (k == 2 ? a.m_y[PV_IDX(i - g.pitch, n_plane, flags)] : a.m_y[i]));
        T sg = (k == 0 || k == 2) ? T(1) : T(-1);
        T rn = d - dj + sg * m;
        T den = v_div(T(1), F.lam_N + sv);
        nl[k] = omb * (F.lam_N * sv * den) + beta * ld_state(Si + (PL_NM + 2 * k) * TILE_PX);
        ne[k] = omb * (F.lam_N * (evn - sv * rn) * den) + beta * ld_state(Si + (PL_NM + 2 * k + 1) * TILE_PX);
        md += nl[k];
        eb[6] += ne[k];
    }

    T alpha = T(0), rph = T(0);
    T J[7];
#pragma unroll
    for (int q = 0; q < 7; ++q) J[q] = T(0);
    unsigned char br = 0;

    // --- a1: photometric factor (Eqs. 2, 3) at the current mean (it enters only
    // the belief below, so it is evaluated after the pairwise messages) ---
    {
        T z = v_exp(d);
        T Xs[3] = {z * (T(u) - g.cx) * g.ifx, z * (T(v) - g.cy) * g.ify, z};
        T Xt[3];
        mat3_vec(R, Xs, Xt);
        Xt[0] += t[0];
        Xt[1] += t[1];
        Xt[2] += t[2];
        T Z = Xt[2];
        bool valid = Z > T(1e-6);
        T iz = valid ? v_div(T(1), Z) : T(0);
        T x = g.fx * Xt[0] * iz + g.cx;
        T y = g.fy * Xt[1] * iz + g.cy;
        // overlap test with a 1e-3 px margin (pixels warped by the identity land on
        // the border exactly); the sample point is clamped into the image
        valid = valid && (x >= T(-1e-3)) && (x <= T(g.W - 1) + T(1e-3)) && (y >= T(-1e-3)) &&
                (y <= T(g.H - 1) + T(1e-3));
        T r = T(0), gx = T(0), gy = T(0);
        if (valid) {
            x = x < T(0) ? T(0) : (x > T(g.W - 1) ? T(g.W - 1) : x);
            y = y < T(0) ? T(0) : (y > T(g.H - 1) ? T(g.H - 1) : y);
            int x0 = (int)v_floor(x), y0 = (int)v_floor(y);
            x0 = min(x0, g.W - 1);
            y0 = min(y0, g.H - 1);
            int x1 = min(x0 + 1, g.W - 1), y1 = min(y0 + 1, g.H - 1);
#ifdef PIXVOD_CHECKED
            if (x0 < 0 || y0 < 0 || (size_t)y1 * g.pitch + x1 >= n_plane) {
                flags |= FLAG_BOUNDS;
                x0 = y0 = x1 = y1 = 0;
            }
#endif
            T ax = x - T(x0), ay = y - T(y0);
            T It = bilinear(a.I_t, g.pitch, x0, y0, x1, y1, ax, ay);
            gx = bilinear(a.g_x, g.pitch, x0, y0, x1, y1, ax, ay);
            gy = bilinear(a.g_y, g.pitch, x0, y0, x1, y1, ax, ay);
            r = a.I_s[i] - It;
            valid = v_finite(r) && v_finite(gx) && v_finite(gy);
        }
        if (valid) {
            // dr/dX_t = -(gx, gy) d(pi)/dX_t
            T a0 = -gx * g.fx * iz, a1 = -gy * g.fy * iz;
            T a2 = (gx * g.fx * Xt[0] + gy * g.fy * Xt[1]) * iz * iz;
            T av[3] = {a0, a1, a2}, b[3];
            mat3T_vec(R, av, b);  // b = R^T a
            J[0] = Xs[1] * b[2] - Xs[2] * b[1];
            J[1] = Xs[2] * b[0] - Xs[0] * b[2];
            J[2] = Xs[0] * b[1] - Xs[1] * b[0];
            J[3] = b[0];
            J[4] = b[1];
            J[5] = b[2];
            J[6] = b[0] * Xs[0] + b[1] * Xs[1] + b[2] * Xs[2];
            T M = v_abs(r) * F.inv_sigma_D;
            const bool hub = M > F.t_huber;
            T w = hub ? v_div(T(2) * F.t_huber * M - F.t_huber * F.t_huber, M * M) : T(1);
            alpha = w * F.lam_D;
            rph = r;
            br = hub ? (BR_VALID | BR_HUBER) : BR_VALID;
        }
    }
    // --- a4: belief, mean update, tangent projection ---
    // With B = blockdiag(M_p, m_d), h = B^-1 eta_o and z = B^-1 J, Sherman-Morrison
    // gives tau = Lambda_b^-1 eta_b = h - z alpha (r + J^T h) / (1 + alpha J^T z),
    // and the marginals of Lambda_b are, with q = J_p^T M_p^-1 J_p,
    //   P = M_p + u u^T,  u = sqrt(alpha m_d / (m_d + alpha J_d^2)) J_p,
    //   s = m_d + alpha J_d^2 / (1 + alpha q),
    // all free of cancellation.
    T tau[7];
    T qv;
    bool ok;
    {
        T Lp[21], idp[6];
#pragma unroll
        for (int q = 0; q < 21; ++q) Lp[q] = Mp[q];
        ok = chol_packed<6>(Lp, idp);
        T up[6], gp[6];
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            up[q] = J[q];
            gp[q] = eb[q];
        }
        fwd_solve<6>(Lp, idp, up);
        bwd_solve<6>(Lp, idp, up);
        fwd_solve<6>(Lp, idp, gp);
        bwd_solve<6>(Lp, idp, gp);
        T jh = T(0);
        qv = T(0);
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            qv += J[q] * up[q];
            jh += J[q] * gp[q];
        }
        const T imd = v_div(T(1), md);
        const T hd = eb[6] * imd;
        const T zd = J[6] * imd;
        const T coef = v_div(alpha * (rph + jh + J[6] * hd), T(1) + alpha * (qv + J[6] * zd));
#pragma unroll
        for (int q = 0; q < 6; ++q) tau[q] = gp[q] - coef * up[q];
        tau[6] = hd - coef * zd;
    }
    bool fin = true;
#pragma unroll
    for (int q = 0; q < 7; ++q) fin = fin && v_finite(tau[q]);
    if (!ok) flags |= FLAG_NONPOS_PIVOT;
    if (!ok || !fin) {
        if (!fin) flags |= FLAG_NONFINITE;
        br |= BR_SKIP;
#pragma unroll
        for (int q = 0; q < 7; ++q) tau[q] = T(0);
    }
    if (a.br) a.br[tile * TILE_PX + tid] = br;
    // mu <- mu (+) tau
    {
        T Rt[9], tt[3], Rn[9], tn[3], xn[6];
        se3_exp(tau, Rt, tt);
        se3_mul(R, t, Rt, tt, Rn, tn);
        se3_log(Rn, tn, xn);
#pragma unroll
        for (int q = 0; q < 6; ++q) Di[q * TILE_PX] = xn[q];
        Di[6 * TILE_PX] = d + tau[6];
    }
    {
        const T bp = v_div(alpha * md, md + alpha * J[6] * J[6]);
        const T sb = v_sqrt(bp);
#pragma unroll
        for (int q = 0; q < 21; ++q) Di[(PL_MP + q) * TILE_PX] = Mp[q];
#pragma unroll
        for (int q = 0; q < 6; ++q) Di[(PL_U + q) * TILE_PX] = sb * J[q];
        Di[PL_S * TILE_PX] = md + v_div(alpha * J[6] * J[6], T(1) + alpha * qv);
    }
    // messages, projected: eta <- eta - Lambda tau
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        Di[(PL_NM + 2 * k) * TILE_PX] = nl[k];
        Di[(PL_NM + 2 * k + 1) * TILE_PX] = ne[k] - nl[k] * tau[6];
    }
#pragma unroll 1
    for (int k = 0; k < 4; ++k) {
        T* mb = msg + (k * ID_STRIDE) * TILE_PX + tid;
        T L[21];
#pragma unroll
        for (int q = 0; q < 21; ++q) L[q] = mb[q * TILE_PX];
#pragma unroll
        for (int r = 0; r < 6; ++r) {
            T e = mb[(21 + r) * TILE_PX];
#pragma unroll
            for (int c = 0; c < 6; ++c) e -= L[pidx(r, c)] * tau[c];
            mb[(21 + r) * TILE_PX] = e;
        }
    }
    if (flags) atomicOr(&a.sc->flags, flags);
    return true;
}

// shared -> global bulk copy by the calling thread, waited for until the writes
// are complete and ordered before the thread's later generic-proxy accesses;
// dst, src and bytes must be multiples of 16 bytes
__device__ __forceinline__ void bulk_copy_s2g(void* dst, const void* src, unsigned bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_u32(src)),
                 "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
    asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

// One synchronous sweep over one state tile (tx, ty) by the calling block (every
// thread of the block must call it). The block must have initialised `bar` (one
// arrival); `parity` is the phase this tile's bulk copy completes. The caller
// synchronises the block before reusing `msg` for another tile. The message
// planes of pixels outside the image are copied through unchanged. Returns
// false (to every thread) when the tile's bulk copy did not arrive within the
// bounded wait: nothing of the tile was stored, FLAG_TIMEOUT is set, and the
// block must take no further tile in this launch.
template <typename T>
__device__ __forceinline__ bool sweep_tile(const SweepArgs<T>& a, int tx, int ty, T* msg, uint64_t* bar,
                                           unsigned parity) {
    const int tid = threadIdx.y * SWEEP_BX + threadIdx.x;
    const size_t tile = (size_t)ty * a.g.tiles_x + tx;
    constexpr unsigned bytes = sizeof(T) * MSG_PLANES * TILE_PX;
    if (tid == 0) {
        // order earlier generic-proxy accesses (global stores of a previous sweep in
        // the same launch, shared-memory use of a previous tile) before the async copy
        asm volatile("fence.proxy.async;" ::: "memory");
        mbar_expect_tx(bar, bytes);
        bulk_copy_g2s(msg, a.in + tile * TILE_WORDS + PL_ID * TILE_PX, bytes, bar);
    }
    const bool ok = sweep_pixel(a, tx, ty, msg, bar, parity);
    // the projected messages written to shared memory (generic proxy) are read by
    // the bulk copy (async proxy): fence, then gather the block; a tile whose
    // messages never arrived is not stored
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    const bool all_ok = __syncthreads_and(ok);
    if (all_ok && tid == 0) bulk_copy_s2g(a.out + tile * TILE_WORDS + PL_ID * TILE_PX, msg, bytes);
    return all_ok;
}

// ---------------------------------------------------------------------------
// a5: pose average (App. C.2) and keyframe anchoring, one launch, fixed order
// ---------------------------------------------------------------------------
constexpr int RED_THREADS = TILE_PX;

// One block per state tile sums that tile's 7 mean planes (double accumulation,
// fixed order); the last block to finish sums the tile partials in tile order,
// writes xi_est and the mean log-depth, composes T_cur = Exp(xi_est) T_kf and,
// at an anchoring frame, moves the keyframe: T_kf <- T_cur, d_prior <- d_mean.
template <typename T>
__device__ __forceinline__ void reduce_tile(const Geometry<T>& g, const T* __restrict__ state,
                                            double* __restrict__ partials, Scalars* sc, int anchor, int tile,
                                            int n_tiles) {
    __shared__ double sh[7][RED_THREADS];
    __shared__ bool last;
    const int tid = threadIdx.x;
    const int u = (tile % g.tiles_x) * TILE_W + tid % TILE_W;
    const int v = (tile / g.tiles_x) * TILE_H + tid / TILE_W;
    double acc[7] = {0, 0, 0, 0, 0, 0, 0};
    if (tid < TILE_PX && u < g.W && v < g.H) {
        const T* st = state + (size_t)tile * TILE_WORDS + tid;
#pragma unroll
        for (int q = 0; q < 7; ++q) acc[q] = double(st[q * TILE_PX]);
    }
#pragma unroll
    for (int q = 0; q < 7; ++q) sh[q][tid] = acc[q];
    __syncthreads();
    for (int s = RED_THREADS / 2; s > 0; s >>= 1) {
        if (tid < s)
#pragma unroll
            for (int q = 0; q < 7; ++q) sh[q][tid] += sh[q][tid + s];
        __syncthreads();
    }
    if (tid == 0) {
#pragma unroll
        for (int q = 0; q < 7; ++q) partials[tile * 7 + q] = sh[q][0];
        __threadfence();
        last = atomicAdd(&sc->counter, 1u) == (unsigned)(n_tiles - 1);
    }
    __syncthreads();
    if (!last) return;
    double r[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int h = tid; h < n_tiles; h += RED_THREADS)
#pragma unroll
        for (int q = 0; q < 7; ++q) r[q] += __ldcg(partials + h * 7 + q);
#pragma unroll
    for (int q = 0; q < 7; ++q) sh[q][tid] = r[q];
    __syncthreads();
    for (int s = RED_THREADS / 2; s > 0; s >>= 1) {
        if (tid < s)
#pragma unroll
            for (int q = 0; q < 7; ++q) sh[q][tid] += sh[q][tid + s];
        __syncthreads();
    }
    if (tid == 0) {
        const double n = double(g.W) * double(g.H);
        double xi[6], R[9], t[3];
        for (int q = 0; q < 6; ++q) {
            xi[q] = sh[q][0] / n;
            sc->xi_est[q] = xi[q];
        }
        sc->d_mean = sh[6][0] / n;
        se3_exp(xi, R, t);
        // T_cur = Exp(xi_est) T_kf with Exp(xi_est) = [R t; 0 1]
        double Tc[16];
        for (int c = 0; c < 4; ++c) {
            for (int r2 = 0; r2 < 3; ++r2)
                Tc[4 * r2 + c] = R[3 * r2] * sc->T_kf[c] + R[3 * r2 + 1] * sc->T_kf[4 + c] +
                                 R[3 * r2 + 2] * sc->T_kf[8 + c] + t[r2] * sc->T_kf[12 + c];
            Tc[12 + c] = sc->T_kf[12 + c];
        }
        for (int q = 0; q < 16; ++q) sc->T_cur[q] = Tc[q];
        if (anchor) {
            for (int q = 0; q < 16; ++q) sc->T_kf[q] = Tc[q];
            sc->d_prior = sc->d_mean;
        }
        sc->counter = 0;
    }
}

template <typename T>
__global__ void __launch_bounds__(RED_THREADS) k_reduce(Geometry<T> g, const T* __restrict__ state,
                                                        double* __restrict__ partials, Scalars* sc,
                                                        int anchor) {
    reduce_tile(g, state, partials, sc, anchor, blockIdx.x, gridDim.x);
}

// Depth output: exp(sign * mu_6) as dense float32.
template <typename T>
__global__ void k_depth_out(Geometry<T> g, const T* __restrict__ state, float* out, T sign) {
    int u = blockIdx.x * blockDim.x + threadIdx.x;
    int v = blockIdx.y * blockDim.y + threadIdx.y;
    if (u >= g.W || v >= g.H) return;
    out[(size_t)v * g.W + u] = float(v_exp(sign * state[state_index(u, v, g.tiles_x) + 6 * TILE_PX]));
}

}  // namespace pv
