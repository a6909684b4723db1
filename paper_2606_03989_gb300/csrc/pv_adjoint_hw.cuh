// Hand-written adjoint of one pixel's sweep update (reverse mode without a tape).
//
// The update of pixel i in one synchronous sweep (Eqs. 2-6 linearised at the
// current mean, the damped factor-to-variable messages, the belief solve, the
// mean update on SE(3) x R and the tangent projection of Sec. 4.1) is a function
// y = F(x) of the values the pixel reads (its own mean and messages, 64 values
// of each neighbour, the source intensity, 12 bilinear taps of I_t, g_x, g_y and
// the factor weights lam_D, 1/sigma_D, lam_N). pixel_vjp recomputes F stage by
// stage and then runs the stages backwards, giving x_bar = (dF/dx)^T y_bar:
//  - the tangent projection eta' = eta - Lambda tau and the outputs P, s;
//  - the belief solve tau = Lambda_b^-1 eta_b with Lambda_b = blockdiag(M_p, m_d)
//    + alpha J J^T: y = M^-1 b has b_bar = M^-1 y_bar and M_bar = -(M^-1 y_bar) y^T,
//    evaluated with the Cholesky factor of M_p (transposed triangular solves);
//  - the photometric factor: the Jacobian J, the Huber weight (the branch the
//    forward took), the warp, and the bilinear gather, whose transpose scatters
//    into the taps;
//  - the normal-integration messages (scalar Schur complements, Eq. 6);
//  - each identity message in its closed Sherman-Morrison form: with
//    C = W + lam_R I + u u^T, Lambda = lam_R C^-1 V = lam_R I - lam_R^2 C^-1 and
//    eta = lam_R C^-1 q, q = eta_v - W r - u (u^T r), so dLambda = lam_R^2 C^-1 dC
//    C^-1 and d eta = lam_R C^-1 (dq - dC C^-1 q) (Eq. 5 through the Schur
//    complement of the 12-D factor + incoming joint);
//  - Exp and Log: their local Jacobians are evaluated by forward-mode dual
//    numbers run through the forward's own code (series or closed form, as the
//    forward took them), so they are the exact derivatives of what the sweep
//    computes: Exp in its 6 inputs, Log in (w, c, t) with w = vee(R - R^T)/2 and
//    c = (tr R - 1)/2, which the Log depends on only.
// Discrete decisions (the warp's validity, the Huber branch, a skipped update)
// are not re-decided: they are taken from the bits the sweep kernel recorded for
// this sweep, so the derivative follows the forward's branch in either precision.
//
// Templated on the arithmetic type (float or double); everything is host- and
// device-compilable.
#pragma once

#include "pv_branch.h"
#include "pv_math.cuh"

namespace pv {
namespace hw {

// the scalar wrappers stay visible next to their dual-number overloads below
using pv::v_abs;
using pv::v_atan2;
using pv::v_div;
using pv::v_exp;
using pv::v_finite;
using pv::v_floor;
using pv::v_rsqrt;
using pv::v_sincos;
using pv::v_sqrt;

// ---------------------------------------------------------------------------
// forward-mode dual numbers (value and N tangents)
// ---------------------------------------------------------------------------
template <typename T, int N>
struct Dual {
    T v;
    T d[N];
    PV_HD Dual() : v(T(0)) {
        for (int i = 0; i < N; ++i) d[i] = T(0);
    }
    PV_HD Dual(double x) : v(T(x)) {
        for (int i = 0; i < N; ++i) d[i] = T(0);
    }
};

template <typename T, int N>
PV_HD Dual<T, N> operator+(const Dual<T, N>& a, const Dual<T, N>& b) {
    Dual<T, N> r;
    r.v = a.v + b.v;
    for (int i = 0; i < N; ++i) r.d[i] = a.d[i] + b.d[i];
    return r;
}
template <typename T, int N>
PV_HD Dual<T, N> operator-(const Dual<T, N>& a, const Dual<T, N>& b) {
    Dual<T, N> r;
    r.v = a.v - b.v;
    for (int i = 0; i < N; ++i) r.d[i] = a.d[i] - b.d[i];
    return r;
}
template <typename T, int N>
PV_HD Dual<T, N> operator-(const Dual<T, N>& a) {
    Dual<T, N> r;
    r.v = -a.v;
    for (int i = 0; i < N; ++i) r.d[i] = -a.d[i];
    return r;
}
template <typename T, int N>
PV_HD Dual<T, N> operator*(const Dual<T, N>& a, const Dual<T, N>& b) {
    Dual<T, N> r;
    r.v = a.v * b.v;
    for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
    return r;
}
// quotient through the forward's own division (approximate for float)
template <typename T, int N>
PV_HD Dual<T, N> v_div(const Dual<T, N>& a, const Dual<T, N>& b) {
    Dual<T, N> r;
    r.v = v_div(a.v, b.v);
    const T ib = T(1) / b.v;
    for (int i = 0; i < N; ++i) r.d[i] = (a.d[i] - r.v * b.d[i]) * ib;
    return r;
}
template <typename T, int N>
PV_HD Dual<T, N> operator/(const Dual<T, N>& a, const Dual<T, N>& b) {
    Dual<T, N> r;
    r.v = a.v / b.v;
    const T ib = T(1) / b.v;
    for (int i = 0; i < N; ++i) r.d[i] = (a.d[i] - r.v * b.d[i]) * ib;
    return r;
}
template <typename T, int N>
PV_HD Dual<T, N>& operator+=(Dual<T, N>& a, const Dual<T, N>& b) { return a = a + b; }
template <typename T, int N>
PV_HD Dual<T, N>& operator-=(Dual<T, N>& a, const Dual<T, N>& b) { return a = a - b; }
template <typename T, int N>
PV_HD Dual<T, N>& operator*=(Dual<T, N>& a, const Dual<T, N>& b) { return a = a * b; }
template <typename T, int N>
PV_HD bool operator<(const Dual<T, N>& a, double b) { return a.v < b; }
template <typename T, int N>
PV_HD bool operator>(const Dual<T, N>& a, double b) { return a.v > b; }
template <typename T, int N>
PV_HD bool operator<(const Dual<T, N>& a, const Dual<T, N>& b) { return a.v < b.v; }
template <typename T, int N>
PV_HD bool operator>(const Dual<T, N>& a, const Dual<T, N>& b) { return a.v > b.v; }

template <typename T, int N>
PV_HD Dual<T, N> chain1(const Dual<T, N>& x, T fv, T dfdx) {
    Dual<T, N> r;
    r.v = fv;
    for (int i = 0; i < N; ++i) r.d[i] = dfdx * x.d[i];
    return r;
}
template <typename T, int N>
PV_HD Dual<T, N> v_sqrt(const Dual<T, N>& x) {
    const T s = v_sqrt(x.v);
    return chain1(x, s, s > T(0) ? T(0.5) / s : T(0));
}
template <typename T, int N>
PV_HD Dual<T, N> v_rsqrt(const Dual<T, N>& x) {
    const T r = v_rsqrt(x.v);
    return chain1(x, r, T(-0.5) * r / x.v);
}
template <typename T, int N>
PV_HD Dual<T, N> v_atan2(const Dual<T, N>& y, const Dual<T, N>& x) {
    Dual<T, N> r;
    r.v = v_atan2(y.v, x.v);
    const T q = T(1) / (x.v * x.v + y.v * y.v);
    for (int i = 0; i < N; ++i) r.d[i] = (x.v * y.d[i] - y.v * x.d[i]) * q;
    return r;
}
template <typename T, int N>
PV_HD void v_sincos(const Dual<T, N>& x, Dual<T, N>* s, Dual<T, N>* c) {
    T sv, cv;
    v_sincos(x.v, &sv, &cv);
    *s = chain1(x, sv, cv);
    *c = chain1(x, cv, -sv);
}

}  // namespace hw

// series limits of a dual number: those of its value type
template <typename T, int N>
struct Prec<hw::Dual<T, N>> : Prec<T> {};

namespace hw {

// ---------------------------------------------------------------------------
// local Jacobians of Exp and Log, contracted with an adjoint
// ---------------------------------------------------------------------------
// xi_bar += (d(R, t)/d xi)^T (R_bar, t_bar) at xi. R depends on theta only and
// t = V(theta) rho, so forward-mode tangents are needed in theta alone:
// rho_bar = V^T t_bar.
template <typename T>
PV_HD void exp_vjp(const T* xi, const T* Rb, const T* tb, T* xib) {
    typedef Dual<T, 3> D;
    D x[6], R[9], t[3], V[9];
    for (int k = 0; k < 6; ++k) {
        x[k] = D(0.0);
        x[k].v = xi[k];
        if (k < 3) x[k].d[k] = T(1);
    }
    se3_exp_V(x, R, t, V);
    for (int k = 0; k < 3; ++k) {
        T acc = T(0);
        for (int q = 0; q < 9; ++q) acc += Rb[q] * R[q].d[k];
        for (int q = 0; q < 3; ++q) acc += tb[q] * t[q].d[k];
        xib[k] += acc;
    }
    for (int k = 0; k < 3; ++k) xib[3 + k] += V[k].v * tb[0] + V[3 + k].v * tb[1] + V[6 + k].v * tb[2];
}

// (R_bar, t_bar) += (d xi / d(R, t))^T xi_bar for xi = Log(R, t). The Log
// depends on R only through w = vee(R - R^T)/2 and c = (tr R - 1)/2, and
// rho = V^-1(theta) t, so forward-mode tangents are needed in (w, c) alone:
// t_bar = V^-T rho_bar.
template <typename T>
PV_HD void log_vjp(const T* R, const T* t, const T* xb, T* Rb, T* tb) {
    typedef Dual<T, 4> D;
    D in[4], tt[3], x[6], Vi[9];
    const T vals[4] = {T(0.5) * (R[7] - R[5]), T(0.5) * (R[2] - R[6]), T(0.5) * (R[3] - R[1]),
                       T(0.5) * (R[0] + R[4] + R[8] - T(1))};
    for (int k = 0; k < 4; ++k) {
        in[k] = D(0.0);
        in[k].v = vals[k];
        in[k].d[k] = T(1);
    }
    for (int k = 0; k < 3; ++k) {
        tt[k] = D(0.0);
        tt[k].v = t[k];
    }
    se3_log_wct(in[0], in[1], in[2], in[3], tt, x, Vi);
    T g[4];
    for (int k = 0; k < 4; ++k) {
        T acc = T(0);
        for (int q = 0; q < 6; ++q) acc += xb[q] * x[q].d[k];
        g[k] = acc;
    }
    // w and c are linear in R
    Rb[7] += T(0.5) * g[0];
    Rb[5] -= T(0.5) * g[0];
    Rb[2] += T(0.5) * g[1];
    Rb[6] -= T(0.5) * g[1];
    Rb[3] += T(0.5) * g[2];
    Rb[1] -= T(0.5) * g[2];
    Rb[0] += T(0.5) * g[3];
    Rb[4] += T(0.5) * g[3];
    Rb[8] += T(0.5) * g[3];
    for (int k = 0; k < 3; ++k) tb[k] += Vi[k].v * xb[3] + Vi[3 + k].v * xb[4] + Vi[6 + k].v * xb[5];
}

// ---------------------------------------------------------------------------
// packed symmetric helpers
// ---------------------------------------------------------------------------
// y = S x for packed symmetric S
template <typename T>
PV_HD void sym_mv(const T* S, const T* x, T* y) {
    for (int r = 0; r < 6; ++r) {
        T acc = T(0);
        for (int c = 0; c < 6; ++c) acc += S[pidx(r, c)] * x[c];
        y[r] = acc;
    }
}
// packed adjoint of a symmetric input M from a matrix adjoint G (full 6x6,
// row-major, not necessarily symmetric): M_bar[p(r,c)] += G_rc + G_cr (r != c),
// G_rr (r == c)
template <typename T>
PV_HD void add_packed_from_full(const T* G, T s, T* Mb) {
    for (int r = 0; r < 6; ++r)
        for (int c = 0; c <= r; ++c) Mb[pidx(r, c)] += s * (r == c ? G[6 * r + r] : G[6 * r + c] + G[6 * c + r]);
}
// packed adjoint of M from the outer product a b^T (as a matrix adjoint)
template <typename T>
PV_HD void add_packed_outer(const T* a, const T* b, T s, T* Mb) {
    for (int r = 0; r < 6; ++r)
        for (int c = 0; c <= r; ++c) Mb[pidx(r, c)] += s * (r == c ? a[r] * b[r] : a[r] * b[c] + a[c] * b[r]);
}
// full symmetric matrix form of a packed adjoint (off-diagonals halved), so that
// <G, dM> = sum_p Mb[p] dM[p] for symmetric dM
template <typename T>
PV_HD void full_from_packed_adjoint(const T* Mb, T* G) {
    for (int r = 0; r < 6; ++r)
        for (int c = 0; c < 6; ++c) G[6 * r + c] = r == c ? Mb[pidx(r, r)] : T(0.5) * Mb[pidx(r, c)];
}

// ---------------------------------------------------------------------------
// per-pixel inputs, context and the vector-Jacobian product
// ---------------------------------------------------------------------------
// values a pixel reads from neighbour j in direction k (slot ko = k ^ 1 at j)
constexpr int NB_XJ = 0;   // mu_j[0:6]
constexpr int NB_DJ = 6;   // mu_j[6]
constexpr int NB_MP = 7;   // M_p,j (21, packed)
constexpr int NB_ML = 28;  // Lambda of j's identity message in slot ko (21)
constexpr int NB_ME = 49;  // eta of that message (6)
constexpr int NB_U = 55;   // u_j (6)
constexpr int NB_S = 61;   // s_j
constexpr int NB_NN = 62;  // j's normal message in slot ko: Lambda
constexpr int NB_NE = 63;  //                                 eta
constexpr int NB_VALS = 64;
constexpr int N_OUT = 151; // output planes, in state order

// What pixel_vjp reads and writes goes through an I/O object `io` (the kernel
// loads from and scatters to device memory, a host check uses arrays):
//   T mu(q), msg(k, q), nm(q)       own mean (7), identity messages (slot k, 27
//                                   values: Lambda packed, eta), normal messages (8)
//   T nb(k, q)                      neighbour value q (NB_*) of direction k
//   T I_s(), tap(q)                 source intensity; I_t, g_x, g_y taps (4 each)
//   T ybar(q)                       adjoint of output plane q (state order)
//   void identity_sums(R, t, L, e)  sums over the directions with a neighbour of
//                                   the damped identity messages (Lambda packed,
//                                   eta) into the pixel at pose (R, t)
//   void identity_eta_adj(w)        sum over them of Lambda_k times the adjoint
//                                   of the projected eta_k' (w_k below)
//   T damped(k, q)                  value q (Lambda packed, eta) of the damped
//                                   message of direction k (with a neighbour)
//   void main_out(p, v), T main_in(p)  what the main stage hands on (plane p,
//                                   MO_*), and that value back
//   void out(q, y, scale)           recomputed output plane q and the magnitude
//                                   of the terms it is formed from (>= 1, >= |y|)
//   void add_mu/add_msg/add_nm/add_nb/add_Is/add_tap(..., v), add_lamD/add_isD/
//        add_lamN(v)                adjoints of the inputs and factor weights
template <typename T>
struct PixCtx {
    T u, v;
    int W, H;
    T fx, fy, cx, cy, ifx, ify;
    bool has[4];      // the neighbour of direction k is in the image
    T m[4];           // normal edge measurement of direction k
    T d_prior, lam_P, lam_Z, lam_R, beta, t_huber;
    T lam_D, inv_sigma_D, lam_N;
    unsigned char br; // recorded decisions (BR_*)
    int x0, y0;       // bilinear cell of the warped point
    bool clamp_x, clamp_y;  // the warped coordinate was clamped into the image
};

// The identity message of direction k (Eq. 5 through the 12-D Schur complement,
// in the sweep kernel's product form), undamped: Lambda_new (packed) and eta_new.
// Also returns what the reverse pass needs: rb, W, the factor L of
// A = W + lam_R I (with 1/L_ii on its diagonal), z = A^-1 u, iuz = 1/(1 + u^T z).
template <typename T>
PV_HD void identity_message(const T* nb, const T* R, const T* t, T lam_R, T* rb, T* W, T* L, T* z, T* iuz_out,
                            T* Lnew, T* enew) {
    {
        T Rj[9], tj[3], Rr[9], tr[3];
        se3_exp(nb + NB_XJ, Rj, tj);
        se3_invmul(Rj, tj, R, t, Rr, tr);
        se3_log(Rr, tr, rb);
    }
    T gv[6], uj[6];
    for (int q = 0; q < 21; ++q) {
        W[q] = nb[NB_MP + q] - nb[NB_ML + q];
        L[q] = W[q];
    }
    for (int q = 0; q < 6; ++q) {
        uj[q] = nb[NB_U + q];
        T wr = T(0);
        for (int c = 0; c < 6; ++c) wr += W[pidx(q, c)] * rb[c];
        gv[q] = -nb[NB_ME + q] - wr;
    }
    for (int q = 0; q < 6; ++q) L[pidx(q, q)] += lam_R;
    T idg[6];
    chol_packed<6>(L, idg);
    for (int q = 0; q < 6; ++q) z[q] = uj[q];
    fwd_solve<6>(L, idg, z);
    bwd_solve<6>(L, idg, z);
    fwd_solve<6>(L, idg, gv);
    bwd_solve<6>(L, idg, gv);
    T uz = T(0), ur = T(0), uh = T(0);
    for (int q = 0; q < 6; ++q) {
        uz += uj[q] * z[q];
        ur += uj[q] * rb[q];
        uh += uj[q] * gv[q];
        L[pidx(q, q)] = idg[q];
    }
    const T iuz = v_div(T(1), T(1) + uz);
    const T crank = lam_R * lam_R * iuz;
    const T ecoef = (ur + uh) * iuz;
    for (int q = 0; q < 6; ++q) enew[q] = lam_R * (gv[q] - ecoef * z[q]);
    for (int c = 0; c < 6; ++c) {
        T x[6];
        for (int r = 0; r < 6; ++r) x[r] = W[pidx(r, c)];
        fwd_solve_id<6>(L, x);
        bwd_solve_id<6>(L, x);
        for (int r = c; r < 6; ++r) Lnew[pidx(r, c)] = lam_R * x[r] + crank * z[r] * z[c];
    }
    *iuz_out = iuz;
}

// C^-1 x with C = A + u u^T, A = L L^T (1/L_ii on the diagonal), z = A^-1 u
template <typename T>
PV_HD void solve_C(const T* L, const T* z, T iuz, const T* u, const T* x, T* y) {
    for (int q = 0; q < 6; ++q) y[q] = x[q];
    fwd_solve_id<6>(L, y);
    bwd_solve_id<6>(L, y);
    T uy = T(0);
    for (int q = 0; q < 6; ++q) uy += u[q] * y[q];
    const T s = uy * iuz;
    for (int q = 0; q < 6; ++q) y[q] -= s * z[q];
}

// Photometric factor (Eqs. 2, 3) at the current mean with the recorded validity
// and Huber branch: J (7), alpha, r. Also the intermediate values the reverse
// pass needs.
template <typename T>
struct Photo {
    T z, Xs[3], Xt[3], iz, x, y, ax, ay, gx, gy, r, a[3], b[3], M, w;
};

template <typename T>
PV_HD void photometric(T d, T I_s, const T* tap, const PixCtx<T>& c, const T* R, const T* t, Photo<T>& P, T* J,
                       T* alpha, T* rph) {
    for (int q = 0; q < 7; ++q) J[q] = T(0);
    *alpha = T(0);
    *rph = T(0);
    P.z = v_exp(d);
    P.Xs[0] = P.z * (c.u - c.cx) * c.ifx;
    P.Xs[1] = P.z * (c.v - c.cy) * c.ify;
    P.Xs[2] = P.z;
    mat3_vec(R, P.Xs, P.Xt);
    P.Xt[0] += t[0];
    P.Xt[1] += t[1];
    P.Xt[2] += t[2];
    if (!(c.br & BR_VALID)) return;
    P.iz = v_div(T(1), P.Xt[2]);
    P.x = c.fx * P.Xt[0] * P.iz + c.cx;
    P.y = c.fy * P.Xt[1] * P.iz + c.cy;
    P.x = P.x < T(0) ? T(0) : (P.x > T(c.W - 1) ? T(c.W - 1) : P.x);
    P.y = P.y < T(0) ? T(0) : (P.y > T(c.H - 1) ? T(c.H - 1) : P.y);
    P.ax = P.x - T(c.x0);
    P.ay = P.y - T(c.y0);
    const T* q = tap;
    const T w00 = (T(1) - P.ax) * (T(1) - P.ay), w10 = P.ax * (T(1) - P.ay);
    const T w01 = (T(1) - P.ax) * P.ay, w11 = P.ax * P.ay;
    const T It = w00 * q[0] + w10 * q[1] + w01 * q[2] + w11 * q[3];
    P.gx = w00 * q[4] + w10 * q[5] + w01 * q[6] + w11 * q[7];
    P.gy = w00 * q[8] + w10 * q[9] + w01 * q[10] + w11 * q[11];
    P.r = I_s - It;
    P.a[0] = -P.gx * c.fx * P.iz;
    P.a[1] = -P.gy * c.fy * P.iz;
    P.a[2] = (P.gx * c.fx * P.Xt[0] + P.gy * c.fy * P.Xt[1]) * P.iz * P.iz;
    mat3T_vec(R, P.a, P.b);
    const T* Xs = P.Xs;
    const T* b = P.b;
    J[0] = Xs[1] * b[2] - Xs[2] * b[1];
    J[1] = Xs[2] * b[0] - Xs[0] * b[2];
    J[2] = Xs[0] * b[1] - Xs[1] * b[0];
    J[3] = b[0];
    J[4] = b[1];
    J[5] = b[2];
    J[6] = b[0] * Xs[0] + b[1] * Xs[1] + b[2] * Xs[2];
    P.M = v_abs(P.r) * c.inv_sigma_D;
    const T th = c.t_huber;
    P.w = (c.br & BR_HUBER) ? v_div(T(2) * th * P.M - th * th, P.M * P.M) : T(1);
    *alpha = P.w * c.lam_D;
    *rph = P.r;
}

// What the reverse pass of an identity message needs from its forward: the
// residual rb, W = M_p,j - Lambda_j->i, C^-1 (packed; C = W + lam_R I + u u^T)
// and eta_new (ID_FWD_VALS values, in this order).
template <typename T>
struct IdFwd {
    T rb[6], W[21], Ci[21], en[6];
};
constexpr int ID_FWD_VALS = 54;

// C^-1 (packed) from the factor of A = W + lam_R I, z = A^-1 u, 1/(1 + u^T z):
// six solves on the unit vectors
template <typename T>
PV_HD void form_Ci(const T* L, const T* z, T iuz, const T* u, T* Ci) {
#pragma unroll
    for (int cc = 0; cc < 6; ++cc) {
        T ec[6], o[6];
        for (int r = 0; r < 6; ++r) ec[r] = r == cc ? T(1) : T(0);
        solve_C(L, z, iuz, u, ec, o);
        for (int r = cc; r < 6; ++r) Ci[pidx(r, cc)] = o[r];
    }
}

// The damped identity message of direction k into the pixel at pose (R, t):
// Lambda (packed) and eta, from the neighbour's values and the pixel's old
// message of slot k; with f, also what its reverse pass needs.
template <typename T, typename IO>
PV_HD void damped_identity(IO& io, const PixCtx<T>& c, int k, const T* R, const T* t, T* L, T* e,
                           IdFwd<T>* f = nullptr) {
    const T beta = c.beta, omb = T(1) - c.beta;
    T nbk[NB_VALS];
    for (int q = 0; q < NB_VALS; ++q) nbk[q] = io.nb(k, q);
    T rb[6], W[21], Lc[21], z[6], iuz, Ln[21], en[6];
    identity_message(nbk, R, t, c.lam_R, rb, W, Lc, z, &iuz, Ln, en);
    for (int q = 0; q < 6; ++q) e[q] = omb * en[q] + beta * io.msg(k, 21 + q);
    for (int q = 0; q < 21; ++q) L[q] = omb * Ln[q] + beta * io.msg(k, q);
    if (f) {
        for (int q = 0; q < 6; ++q) {
            f->rb[q] = rb[q];
            f->en[q] = en[q];
        }
        for (int q = 0; q < 21; ++q) f->W[q] = W[q];
        form_Ci(Lc, z, iuz, nbk + NB_U, f->Ci);
    }
}

// The adjoint of the projected eta_k' = eta_k - Lambda_k tau reaches tau as
// -Lambda_k ybar(eta_k'): w_k = Lambda_k ybar(eta_k') (an I/O object's
// identity_eta_adj sums it over the directions). identity_sums_direct computes
// both sums from the damped messages (for an I/O object without a forward stage
// of its own).
template <typename T, typename IO>
PV_HD void identity_w(IO& io, int k, const T* L, T* w) {
    T eyb[6];
    for (int r = 0; r < 6; ++r) eyb[r] = io.ybar(35 + 27 * k + 21 + r);
    sym_mv(L, eyb, w);
}

template <typename T, typename IO>
PV_HD void identity_sums_direct(IO& io, const PixCtx<T>& c, const T* R, const T* t, T* Ls, T* es, T* ws) {
    for (int q = 0; q < 21; ++q) Ls[q] = T(0);
    for (int q = 0; q < 6; ++q) es[q] = ws[q] = T(0);
    for (int k = 0; k < 4; ++k) {
        if (!c.has[k]) continue;
        T L[21], e[6], w[6];
        damped_identity(io, c, k, R, t, L, e);
        identity_w(io, k, L, w);
        for (int q = 0; q < 21; ++q) Ls[q] += L[q];
        for (int q = 0; q < 6; ++q) {
            es[q] += e[q];
            ws[q] += w[q];
        }
    }
}

// What the main stage of the reverse pass hands to the per-direction and pose
// stages (planes of io.main_out): the update tau and the adjoints of M_p and of
// eta_b (from which each direction forms its damped message's adjoint), of the
// pixel's rotation and translation (R, t = Exp(xi)), of xi through the prior, and
// of the log-depth.
constexpr int MO_TAU = 0, MO_MPB = 7, MO_EBB = 28, MO_RB = 34, MO_TB = 43, MO_XIB = 46, MO_DB = 52;
constexpr int MO_PLANES = 53;

// Main stage: the update's outputs but the identity messages' (through io.out),
// and the reverse pass of everything but the identity messages and the final
// Exp(xi); the adjoints of the inputs it reaches go through io.add_*, the rest
// through io.main_out. The damped identity messages enter only as their sums.
template <typename T, typename IO>
PV_HD void pixel_vjp_main(IO& io, const PixCtx<T>& c) {
    const T lam_R = c.lam_R, beta = c.beta, omb = T(1) - c.beta;
    // ---------------- forward ----------------
    T xi[6];
    for (int q = 0; q < 6; ++q) xi[q] = io.mu(q);
    const T d = io.mu(6);
    T R[9], t[3];
    se3_exp(xi, R, t);
    T eb[7], Mp[21];
    for (int q = 0; q < 7; ++q) eb[q] = T(0);
    for (int q = 0; q < 21; ++q) Mp[q] = T(0);
    for (int k = 0; k < 6; ++k) {
        Mp[pidx(k, k)] = c.lam_P;
        eb[k] -= c.lam_P * xi[k];
    }
    T md = c.lam_Z;
    eb[6] -= c.lam_Z * (d - c.d_prior);
    {
        T Ls[21], es[6];  // the damped identity messages, summed
        io.identity_sums(R, t, Ls, es);
        for (int q = 0; q < 6; ++q) eb[q] += es[q];
        for (int q = 0; q < 21; ++q) Mp[q] += Ls[q];
    }
    T nl[4], ne[4];
    for (int k = 0; k < 4; ++k) {
        nl[k] = T(0);
        ne[k] = T(0);
        if (!c.has[k]) continue;
        const T sv = io.nb(k, NB_S) - io.nb(k, NB_NN);
        const T evn = -io.nb(k, NB_NE);
        const T sg = (k == 0 || k == 2) ? T(1) : T(-1);
        const T rn = d - io.nb(k, NB_DJ) + sg * c.m[k];
        const T den = v_div(T(1), c.lam_N + sv);
        nl[k] = omb * (c.lam_N * sv * den) + beta * io.nm(2 * k);
        ne[k] = omb * (c.lam_N * (evn - sv * rn) * den) + beta * io.nm(2 * k + 1);
        md += nl[k];
        eb[6] += ne[k];
    }
    Photo<T> P;
    T J[7], alpha, rph, tap[12];
    for (int q = 0; q < 12; ++q) tap[q] = io.tap(q);
    const T I_s = io.I_s();
    photometric(d, I_s, tap, c, R, t, P, J, &alpha, &rph);
    // belief solve
    T Lp[21], idp[6], up[6], gp[6];
    for (int q = 0; q < 21; ++q) Lp[q] = Mp[q];
    chol_packed<6>(Lp, idp);
    for (int q = 0; q < 6; ++q) {
        up[q] = J[q];
        gp[q] = eb[q];
    }
    fwd_solve<6>(Lp, idp, up);
    bwd_solve<6>(Lp, idp, up);
    fwd_solve<6>(Lp, idp, gp);
    bwd_solve<6>(Lp, idp, gp);
    T qv = T(0), jh = T(0);
    for (int q = 0; q < 6; ++q) {
        qv += J[q] * up[q];
        jh += J[q] * gp[q];
    }
    const T imd = v_div(T(1), md);
    const T hd = eb[6] * imd;
    const T zd = J[6] * imd;
    const T num = alpha * (rph + jh + J[6] * hd);
    const T dnm = T(1) + alpha * (qv + J[6] * zd);
    const T coef = v_div(num, dnm);
    const bool skip = (c.br & BR_SKIP) != 0;
    T tau[7];
    for (int q = 0; q < 6; ++q) tau[q] = skip ? T(0) : gp[q] - coef * up[q];
    tau[6] = skip ? T(0) : hd - coef * zd;
    // outputs
    T Rt[9], tt[3], Rn[9], tn[3];
    se3_exp(tau, Rt, tt);
    se3_mul(R, t, Rt, tt, Rn, tn);
    {
        T xn[6];
        se3_log(Rn, tn, xn);
        for (int q = 0; q < 6; ++q) io.out(q, xn[q], v_abs(xn[q]) > T(1) ? v_abs(xn[q]) : T(1));
    }
    const T dn = d + tau[6];
    io.out(6, dn, v_abs(dn) > T(1) ? v_abs(dn) : T(1));
    const T dd = md + alpha * J[6] * J[6];
    const T bp = v_div(alpha * md, dd);
    const T sb = v_sqrt(bp);
    const T es = T(1) + alpha * qv;
    auto out_plain = [&](int q, T y) { io.out(q, y, v_abs(y) > T(1) ? v_abs(y) : T(1)); };
    for (int q = 0; q < 21; ++q) out_plain(7 + q, Mp[q]);
    for (int q = 0; q < 6; ++q) out_plain(28 + q, sb * J[q]);
    out_plain(34, md + v_div(alpha * J[6] * J[6], es));
    for (int k = 0; k < 4; ++k) {
        out_plain(143 + 2 * k, nl[k]);
        const T e = ne[k] - nl[k] * tau[6];
        const T m = v_abs(ne[k]) + v_abs(nl[k] * tau[6]);
        io.out(144 + 2 * k, e, m > v_abs(e) ? (m > T(1) ? m : T(1)) : (v_abs(e) > T(1) ? v_abs(e) : T(1)));
    }

    // ---------------- reverse ----------------
    T taub[7], Mpb[21], ebb[7], mdb, Jb[7], alphab = T(0), rphb = T(0), Rb[9], tb[3], db;
    for (int q = 0; q < 7; ++q) {
        taub[q] = T(0);
        ebb[q] = T(0);
        Jb[q] = T(0);
    }
    for (int q = 0; q < 9; ++q) Rb[q] = T(0);
    for (int q = 0; q < 3; ++q) tb[q] = T(0);
    // projected messages eta' = eta - Lambda tau (the adjoints of the damped
    // messages themselves are formed per direction), and the normal ones
    {
        T ws[6];
        io.identity_eta_adj(ws);
        for (int q = 0; q < 6; ++q) taub[q] -= ws[q];
    }
    T nlb[4], neb[4];
    for (int k = 0; k < 4; ++k) {
        const T nyb = io.ybar(143 + 2 * k), eyn = io.ybar(144 + 2 * k);
        nlb[k] = nyb - eyn * tau[6];
        neb[k] = eyn;
        taub[6] -= nl[k] * eyn;
    }
    // s' = md + alpha J6^2 / es
    const T syb = io.ybar(34);
    mdb = syb;
    const T ies = T(1) / es;
    alphab += syb * J[6] * J[6] * ies * ies;
    Jb[6] += syb * T(2) * alpha * J[6] * ies;
    T qvb = -syb * alpha * alpha * J[6] * J[6] * ies * ies;
    // u' = sb J_p
    {
        T sbb = T(0);
        for (int q = 0; q < 6; ++q) {
            const T uyb = io.ybar(28 + q);
            Jb[q] += sb * uyb;
            sbb += J[q] * uyb;
        }
        if (sb > T(0)) {
            const T bpb = sbb * T(0.5) / sb;
            const T idd = T(1) / dd;
            alphab += bpb * md * md * idd * idd;
            mdb += bpb * alpha * alpha * J[6] * J[6] * idd * idd;
            Jb[6] -= bpb * T(2) * alpha * alpha * md * J[6] * idd * idd;
        }
    }
    // Mp' = Mp
    for (int q = 0; q < 21; ++q) Mpb[q] = io.ybar(7 + q);
    // mean update: y[0:6] = Log(Exp(xi) Exp(tau_p)), y[6] = d + tau_6
    db = io.ybar(6);
    taub[6] += db;
    {
        T xnb[6], Rnb[9], tnb[3], Rtb[9], ttb[3];
        for (int q = 0; q < 6; ++q) xnb[q] = io.ybar(q);
        for (int q = 0; q < 9; ++q) Rnb[q] = T(0);
        for (int q = 0; q < 3; ++q) tnb[q] = T(0);
        log_vjp(Rn, tn, xnb, Rnb, tnb);
        // Rn = R Rt, tn = R tt + t
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                T a1 = T(0), a2 = T(0);
                for (int m = 0; m < 3; ++m) {
                    a1 += Rnb[3 * i + m] * Rt[3 * j + m];  // (Rn_bar Rt^T)_ij
                    a2 += R[3 * m + i] * Rnb[3 * m + j];   // (R^T Rn_bar)_ij
                }
                Rb[3 * i + j] += a1 + tnb[i] * tt[j];
                Rtb[3 * i + j] = a2;
            }
        for (int j = 0; j < 3; ++j) {
            ttb[j] = R[j] * tnb[0] + R[3 + j] * tnb[1] + R[6 + j] * tnb[2];
            tb[j] += tnb[j];
        }
        if (!skip) exp_vjp(tau, Rtb, ttb, taub);
    }
    // belief solve (tau); with skip, tau = 0 and qv reaches s' only
    {
        T gpb[6], upb[6];
        for (int q = 0; q < 6; ++q) {
            gpb[q] = skip ? T(0) : taub[q];
            upb[q] = skip ? T(0) : -coef * taub[q];
        }
        if (!skip) {
            T coefb = -taub[6] * zd;
            for (int q = 0; q < 6; ++q) coefb -= taub[q] * up[q];
            T hdb = taub[6], zdb = -coef * taub[6];
            const T idn = T(1) / dnm;
            const T numb = coefb * idn, dnmb = -coefb * coef * idn;
            alphab += numb * (rph + jh + J[6] * hd) + dnmb * (qv + J[6] * zd);
            rphb += numb * alpha;
            const T jhb = numb * alpha;
            Jb[6] += numb * alpha * hd + dnmb * alpha * zd;
            hdb += numb * alpha * J[6];
            qvb += dnmb * alpha;
            zdb += dnmb * alpha * J[6];
            ebb[6] += hdb * imd;
            const T imdb = hdb * eb[6] + zdb * J[6];
            Jb[6] += zdb * imd;
            mdb -= imdb * imd * imd;
            for (int q = 0; q < 6; ++q) {
                Jb[q] += jhb * gp[q];
                gpb[q] += jhb * J[q];
            }
        }
        for (int q = 0; q < 6; ++q) {
            Jb[q] += qvb * up[q];
            upb[q] += qvb * J[q];
        }
        // up = Mp^-1 J_p, gp = Mp^-1 eb_p
        fwd_solve<6>(Lp, idp, upb);
        bwd_solve<6>(Lp, idp, upb);
        for (int q = 0; q < 6; ++q) Jb[q] += upb[q];
        add_packed_outer(upb, up, T(-1), Mpb);
        if (!skip) {
            fwd_solve<6>(Lp, idp, gpb);
            bwd_solve<6>(Lp, idp, gpb);
            for (int q = 0; q < 6; ++q) ebb[q] += gpb[q];
            add_packed_outer(gpb, gp, T(-1), Mpb);
        }
    }
    // photometric factor
    if (c.br & BR_VALID) {
        const T wb = alphab * c.lam_D;
        io.add_lamD(alphab * P.w);
        T rb_ = rphb;
        if (c.br & BR_HUBER) {
            const T th = c.t_huber, M = P.M;
            const T dwdM = -T(2) * th / (M * M) + T(2) * th * th / (M * M * M);
            const T Mb = wb * dwdM;
            const T sgn = P.r < T(0) ? T(-1) : T(1);
            rb_ += Mb * sgn * c.inv_sigma_D;
            io.add_isD(Mb * v_abs(P.r));
        }
        // J from Xs and b
        T bb[3], Xsb[3];
        const T* Xs = P.Xs;
        const T* b = P.b;
        const T cb[3] = {Jb[0], Jb[1], Jb[2]};
        bb[0] = Jb[3] + Jb[6] * Xs[0] + (cb[1] * Xs[2] - cb[2] * Xs[1]);
        bb[1] = Jb[4] + Jb[6] * Xs[1] + (cb[2] * Xs[0] - cb[0] * Xs[2]);
        bb[2] = Jb[5] + Jb[6] * Xs[2] + (cb[0] * Xs[1] - cb[1] * Xs[0]);
        Xsb[0] = Jb[6] * b[0] + (b[1] * cb[2] - b[2] * cb[1]);
        Xsb[1] = Jb[6] * b[1] + (b[2] * cb[0] - b[0] * cb[2]);
        Xsb[2] = Jb[6] * b[2] + (b[0] * cb[1] - b[1] * cb[0]);
        // b = R^T a
        T ab[3];
        mat3_vec(R, bb, ab);
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) Rb[3 * i + j] += P.a[i] * bb[j];
        // a from gx, gy, Xt, iz
        const T iz = P.iz;
        const T gxb = -ab[0] * c.fx * iz + ab[2] * c.fx * P.Xt[0] * iz * iz;
        const T gyb = -ab[1] * c.fy * iz + ab[2] * c.fy * P.Xt[1] * iz * iz;
        T Xtb[3] = {ab[2] * P.gx * c.fx * iz * iz, ab[2] * P.gy * c.fy * iz * iz, T(0)};
        T izb = -ab[0] * P.gx * c.fx - ab[1] * P.gy * c.fy +
                ab[2] * (P.gx * c.fx * P.Xt[0] + P.gy * c.fy * P.Xt[1]) * T(2) * iz;
        // r = I_s - It
        io.add_Is(rb_);
        const T Itb = -rb_;
        const T ax = P.ax, ay = P.ay;
        const T w00 = (T(1) - ax) * (T(1) - ay), w10 = ax * (T(1) - ay), w01 = (T(1) - ax) * ay, w11 = ax * ay;
        const T img_b[3] = {Itb, gxb, gyb};
        T axb = T(0), ayb = T(0);
        for (int m = 0; m < 3; ++m) {
            const T* q = tap + 4 * m;
            io.add_tap(4 * m + 0, w00 * img_b[m]);
            io.add_tap(4 * m + 1, w10 * img_b[m]);
            io.add_tap(4 * m + 2, w01 * img_b[m]);
            io.add_tap(4 * m + 3, w11 * img_b[m]);
            axb += img_b[m] * ((T(1) - ay) * (q[1] - q[0]) + ay * (q[3] - q[2]));
            ayb += img_b[m] * (((T(1) - ax) * q[2] + ax * q[3]) - ((T(1) - ax) * q[0] + ax * q[1]));
        }
        // x = fx Xt0 iz + cx (clamped: no derivative), likewise y
        if (!c.clamp_x) {
            Xtb[0] += axb * c.fx * iz;
            izb += axb * c.fx * P.Xt[0];
        }
        if (!c.clamp_y) {
            Xtb[1] += ayb * c.fy * iz;
            izb += ayb * c.fy * P.Xt[1];
        }
        Xtb[2] -= izb * iz * iz;
        // Xt = R Xs + t
        for (int i = 0; i < 3; ++i) {
            tb[i] += Xtb[i];
            for (int j = 0; j < 3; ++j) {
                Rb[3 * i + j] += Xtb[i] * Xs[j];
                Xsb[j] += R[3 * i + j] * Xtb[i];
            }
        }
        // Xs = z (pu, pv, 1), z = exp(d)
        const T zb = Xsb[0] * (c.u - c.cx) * c.ifx + Xsb[1] * (c.v - c.cy) * c.ify + Xsb[2];
        db += zb * P.z;
    }
    // messages enter M_p and eta_b; priors: eb_p = -lam_P xi + ..., eb_6 =
    // -lam_Z (d - d_prior) + ...
    T xib[6];
    for (int q = 0; q < 6; ++q) xib[q] = -c.lam_P * ebb[q];
    db -= c.lam_Z * ebb[6];
    // normal-integration messages
    T lamNb = T(0);
    for (int k = 0; k < 4; ++k) {
        if (!c.has[k]) continue;
        const T nlk = nlb[k] + mdb, nek = neb[k] + ebb[6];
        const T sj = io.nb(k, NB_S), nn = io.nb(k, NB_NN);
        const T sv = sj - nn;
        const T evn = -io.nb(k, NB_NE);
        const T sg = (k == 0 || k == 2) ? T(1) : T(-1);
        const T rn = d - io.nb(k, NB_DJ) + sg * c.m[k];
        const T lN = c.lam_N;
        const T den = T(1) / (lN + sv);
        const T qn = evn - sv * rn;
        io.add_nm(2 * k, beta * nlk);
        io.add_nm(2 * k + 1, beta * nek);
        const T a = omb * nlk, e = omb * nek;
        const T svb = a * lN * lN * den * den + e * (-lN * qn * den * den - lN * den * rn);
        lamNb += a * sv * sv * den * den + e * qn * sv * den * den;
        const T evnb = e * lN * den;
        const T rnb = -e * lN * den * sv;
        io.add_nb(k, NB_S, svb);
        io.add_nb(k, NB_NN, -svb);
        io.add_nb(k, NB_NE, -evnb);
        db += rnb;
        io.add_nb(k, NB_DJ, -rnb);
    }
    io.add_lamN(lamNb);
    for (int q = 0; q < 7; ++q) io.main_out(MO_TAU + q, tau[q]);
    for (int q = 0; q < 21; ++q) io.main_out(MO_MPB + q, Mpb[q]);
    for (int q = 0; q < 6; ++q) io.main_out(MO_EBB + q, ebb[q]);
    for (int q = 0; q < 9; ++q) io.main_out(MO_RB + q, Rb[q]);
    for (int q = 0; q < 3; ++q) io.main_out(MO_TB + q, tb[q]);
    for (int q = 0; q < 6; ++q) io.main_out(MO_XIB + q, xib[q]);
    io.main_out(MO_DB, db);
}

// Row r of a projected identity message, eta_r' = eta_r - sum_c Lambda_rc tau_c
// (Lrow: Lambda_r0 .. Lambda_r5), and the magnitude of the terms it is formed
// from, as the recompute check's scale (>= 1, >= |eta_r'|).
template <typename T>
PV_HD void projected_eta_row(const T* Lrow, T er, const T* tau, T* y, T* scale) {
    T e = er, m = v_abs(er);
    for (int cc = 0; cc < 6; ++cc) {
        e -= Lrow[cc] * tau[cc];
        m += v_abs(Lrow[cc] * tau[cc]);
    }
    *y = e;
    *scale = m > v_abs(e) ? (m > T(1) ? m : T(1)) : (v_abs(e) > T(1) ? v_abs(e) : T(1));
}

// The outputs of the damped identity message of direction k (Lambda' = Lambda,
// eta' = eta - Lambda tau; zero without a neighbour), through io.out.
template <typename T, typename IO>
PV_HD void identity_outputs(IO& io, const PixCtx<T>& c, int k, const T* tau) {
    T L[21], el[6];
    for (int q = 0; q < 21; ++q) L[q] = c.has[k] ? io.damped(k, q) : T(0);
    for (int q = 0; q < 6; ++q) el[q] = c.has[k] ? io.damped(k, 21 + q) : T(0);
    for (int q = 0; q < 21; ++q) io.out(35 + 27 * k + q, L[q], v_abs(L[q]) > T(1) ? v_abs(L[q]) : T(1));
    for (int r = 0; r < 6; ++r) {
        T Lrow[6], y, sc;
        for (int cc = 0; cc < 6; ++cc) Lrow[cc] = L[pidx(r, cc)];
        projected_eta_row(Lrow, el[r], tau, &y, &sc);
        io.out(35 + 27 * k + 21 + r, y, sc);
    }
}

// The adjoint of the damped identity message of direction k (Lbar packed, ebar)
// from those of its outputs and of M_p and eta_b (Mpb, ebb); the pixel's own old
// message of slot k enters it (damping) through io.add_msg.
template <typename T, typename IO>
PV_HD void identity_msg_adjoint(IO& io, const PixCtx<T>& c, int k, const T* tau, const T* Mpb, const T* ebb, T* Lb,
                                T* eb) {
    T eyb[6];
    for (int q = 0; q < 21; ++q) Lb[q] = io.ybar(35 + 27 * k + q);
    for (int r = 0; r < 6; ++r) eyb[r] = io.ybar(35 + 27 * k + 21 + r);
    add_packed_outer(eyb, tau, T(-1), Lb);
    for (int q = 0; q < 21; ++q) {
        Lb[q] += Mpb[q];
        io.add_msg(k, q, c.beta * Lb[q]);
    }
    for (int q = 0; q < 6; ++q) {
        eb[q] = eyb[q] + ebb[q];
        io.add_msg(k, 21 + q, c.beta * eb[q]);
    }
}

// Per-direction stage: the reverse pass of the identity message of direction k
// (Eq. 5 through the Schur complement) at the pixel's pose (R, t), given the
// adjoints of its damped value (Lbar packed, ebar); adds the adjoints of the
// neighbour's values through io.add_nb and the pose's to (Rb, tb).
template <typename T, typename IO>
PV_HD void identity_vjp(IO& io, const PixCtx<T>& c, int k, const T* R, const T* t, const IdFwd<T>& f,
                        const T* Lbar, const T* ebar, T* Rb, T* tb) {
    const T lam_R = c.lam_R, omb = T(1) - c.beta;
    const T* rb = f.rb;
    const T* W = f.W;
    const T* Ci = f.Ci;
    T uj[6], xj[6];
    for (int q = 0; q < 6; ++q) {
        uj[q] = io.nb(k, NB_U + q);
        xj[q] = io.nb(k, NB_XJ + q);
    }
    // y = C^-1 q = eta_new / lam_R; w = lam_R C^-1 eta_new_bar
    T yv[6], wv[6], eb_[6];
    for (int q = 0; q < 6; ++q) {
        yv[q] = f.en[q] / lam_R;
        eb_[q] = omb * ebar[q];
    }
    sym_mv(Ci, eb_, wv);
    for (int q = 0; q < 6; ++q) wv[q] *= lam_R;
    // C_bar = lam_R^2 C^-1 G C^-1 - w y^T, G the symmetric matrix form of the
    // adjoint of Lambda (off-diagonals halved). Only C_bar + C_bar^T reaches W
    // (W_bar[p(r,c)] = C_bar_rc + C_bar_cr, diagonal C_bar_rr) and u (u_bar =
    // (C_bar + C_bar^T) u). M = C^-1 G C^-1 is symmetric: formed column by
    // column.
    T M[21];
    {
        T Gp[21];
        for (int r = 0; r < 6; ++r)
            for (int c2 = 0; c2 <= r; ++c2) Gp[pidx(r, c2)] = (r == c2 ? omb : T(0.5) * omb) * Lbar[pidx(r, c2)];
#pragma unroll
        for (int cc = 0; cc < 6; ++cc) {
            T P[6];  // column cc of G C^-1
            for (int a = 0; a < 6; ++a) {
                T acc = T(0);
                for (int b = 0; b < 6; ++b) acc += Gp[pidx(a, b)] * Ci[pidx(b, cc)];
                P[a] = acc;
            }
            for (int r = cc; r < 6; ++r) {
                T acc = T(0);
                for (int a = 0; a < 6; ++a) acc += Ci[pidx(r, a)] * P[a];
                M[pidx(r, cc)] = acc;
            }
        }
    }
    T Wb[21], ub[6];
    for (int r = 0; r < 6; ++r) ub[r] = T(0);
    {
        const T l2 = lam_R * lam_R;
#pragma unroll
        for (int r = 0; r < 6; ++r)
            for (int c2 = 0; c2 <= r; ++c2) {
                const T sc = T(2) * l2 * M[pidx(r, c2)] - (wv[r] * yv[c2] + wv[c2] * yv[r]);  // C_bar_rc + C_bar_cr
                Wb[pidx(r, c2)] = r == c2 ? T(0.5) * sc : sc;
                ub[r] += sc * uj[c2];
                if (r != c2) ub[c2] += sc * uj[r];
            }
    }
    // q = g0 - u (u^T rb), g0 = -eta_J - W rb; q_bar = w
    T urb = T(0), uw = T(0);
    for (int q = 0; q < 6; ++q) {
        urb += uj[q] * rb[q];
        uw += uj[q] * wv[q];
    }
    T rbb[6], Ww[6];
    sym_mv(W, wv, Ww);
    for (int q = 0; q < 6; ++q) {
        ub[q] -= wv[q] * urb + rb[q] * uw;
        rbb[q] = -uj[q] * uw - Ww[q];
        io.add_nb(k, NB_ME + q, -wv[q]);
    }
    add_packed_outer(wv, rb, T(-1), Wb);
    for (int q = 0; q < 6; ++q) io.add_nb(k, NB_U + q, ub[q]);
    for (int q = 0; q < 21; ++q) {
        io.add_nb(k, NB_MP + q, Wb[q]);
        io.add_nb(k, NB_ML + q, -Wb[q]);
    }
    // rb = Log(Exp(xi_j)^-1 Exp(xi_i))
    T Rj[9], tj[3], Rr[9], tr[3];
    se3_exp(xj, Rj, tj);
    se3_invmul(Rj, tj, R, t, Rr, tr);
    T Rrb[9], trb[3];
    for (int q = 0; q < 9; ++q) Rrb[q] = T(0);
    for (int q = 0; q < 3; ++q) trb[q] = T(0);
    log_vjp(Rr, tr, rbb, Rrb, trb);
    // Rr = Rj^T R, tr = Rj^T (t - tj)
    T Rjb[9], tjb[3];
    const T dl[3] = {t[0] - tj[0], t[1] - tj[1], t[2] - tj[2]};
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            T a1 = T(0), a2 = T(0);
            for (int m = 0; m < 3; ++m) {
                a1 += R[3 * i + m] * Rrb[3 * j + m];   // (R Rr_bar^T)_ij
                a2 += Rj[3 * i + m] * Rrb[3 * m + j];  // (Rj Rr_bar)_ij
            }
            Rjb[3 * i + j] = a1 + dl[i] * trb[j];
            Rb[3 * i + j] += a2;
        }
    for (int i = 0; i < 3; ++i) {
        const T v = Rj[3 * i] * trb[0] + Rj[3 * i + 1] * trb[1] + Rj[3 * i + 2] * trb[2];
        tb[i] += v;
        tjb[i] = -v;
    }
    T xjb[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
    exp_vjp(xj, Rjb, tjb, xjb);
    for (int q = 0; q < 6; ++q) io.add_nb(k, NB_XJ + q, xjb[q]);
}

// Pose stage: xi_bar from the accumulated (R_bar, t_bar) of Exp(xi), plus the
// prior's part, and the log-depth's adjoint.
template <typename T, typename IO>
PV_HD void pose_vjp(IO& io, const T* xi, const T* Rb, const T* tb, const T* xib_in, T db) {
    T xib[6];
    for (int q = 0; q < 6; ++q) xib[q] = xib_in[q];
    exp_vjp(xi, Rb, tb, xib);
    for (int q = 0; q < 6; ++q) io.add_mu(q, xib[q]);
    io.add_mu(6, db);
}

// The whole reverse pass of one pixel in one thread: the update's outputs
// (through io.out) and the adjoints of its inputs (through io.add_*) for the
// output adjoints io.ybar.
template <typename T, typename IO>
PV_HD void pixel_vjp(IO& io, const PixCtx<T>& c) {
    pixel_vjp_main(io, c);
    T xi[6], R[9], t[3], Rb[9], tb[3], xib[6], tau[7], Mpb[21], ebb[6];
    for (int q = 0; q < 6; ++q) xi[q] = io.mu(q);
    se3_exp(xi, R, t);
    for (int q = 0; q < 7; ++q) tau[q] = io.main_in(MO_TAU + q);
    for (int q = 0; q < 21; ++q) Mpb[q] = io.main_in(MO_MPB + q);
    for (int q = 0; q < 6; ++q) ebb[q] = io.main_in(MO_EBB + q);
    for (int q = 0; q < 9; ++q) Rb[q] = io.main_in(MO_RB + q);
    for (int q = 0; q < 3; ++q) tb[q] = io.main_in(MO_TB + q);
    for (int q = 0; q < 6; ++q) xib[q] = io.main_in(MO_XIB + q);
    for (int k = 0; k < 4; ++k) {
        identity_outputs(io, c, k, tau);
        if (!c.has[k]) continue;
        T Lb[21], eb[6], Ld[21], ed[6];
        IdFwd<T> f;
        damped_identity(io, c, k, R, t, Ld, ed, &f);
        identity_msg_adjoint(io, c, k, tau, Mpb, ebb, Lb, eb);
        identity_vjp(io, c, k, R, t, f, Lb, eb, Rb, tb);
    }
    pose_vjp(io, xi, Rb, tb, xib, io.main_in(MO_DB));
}

}  // namespace hw
}  // namespace pv
