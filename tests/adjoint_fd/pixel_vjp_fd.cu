// Host check of the hand-written reverse pass of one pixel's sweep update
// (hw::pixel_vjp, FP64) against central finite differences of the same forward:
// for a random output adjoint ybar, the gradient of L = <ybar, update(inputs)>
// with respect to every input (own mean and old messages, normal messages, the
// 64 values read from each neighbour, source intensity, the 12 bilinear taps,
// the three factor weights) must match (L(x + h) - L(x - h)) / 2h.
// Host code only (no kernels): built with nvcc for the __host__ __device__
// functions, run on the CPU.
//
//   pixel_vjp_fd <huber 0|1> <case 0|1|2>
//     case 0: interior pixel, update applied; 1: update skipped (recorded
//     BR_SKIP); 2: border pixel (left and upper neighbours missing)
//
// Prints one line: "inputs N nonzero G mismatches M worst W".
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <random>
#include <vector>

#include "pv_adjoint_hw.cuh"

using namespace pv;
using namespace pv::hw;
typedef double T;

// every input of one pixel's update, flat (the finite differences walk it)
struct PixIn {
    T mu[7], msg[108], nm[8], nb[4][NB_VALS], I_s, tap[12], lam_D, inv_sigma_D, lam_N;
};

// the I/O object of hw::pixel_vjp on host arrays; the damped identity messages
// and the main stage's hand-over are kept in the object (a batch of one pixel)
struct HostIO {
    const PixIn* in;
    PixIn* xb;
    const T* yb;
    T* y;
    const PixCtx<T>* c;
    T fwd[4][27], ws[6], mo[MO_PLANES];

    __host__ __device__ void identity_sums(const T* R, const T* t, T* Ls, T* es) {
        identity_sums_direct(*this, *c, R, t, Ls, es, ws);
        for (int k = 0; k < 4; ++k) {
            if (!c->has[k]) continue;
            T L[21], e[6];
            damped_identity(*this, *c, k, R, t, L, e);
            for (int q = 0; q < 21; ++q) fwd[k][q] = L[q];
            for (int q = 0; q < 6; ++q) fwd[k][21 + q] = e[q];
        }
    }
    __host__ __device__ void identity_eta_adj(T* w) const {
        for (int q = 0; q < 6; ++q) w[q] = ws[q];
    }
    __host__ __device__ T damped(int k, int q) const { return fwd[k][q]; }
    __host__ __device__ void main_out(int p, T v) { mo[p] = v; }
    __host__ __device__ T main_in(int p) const { return mo[p]; }
    __host__ __device__ T mu(int q) const { return in->mu[q]; }
    __host__ __device__ T msg(int k, int q) const { return in->msg[27 * k + q]; }
    __host__ __device__ T nm(int q) const { return in->nm[q]; }
    __host__ __device__ T nb(int k, int q) const { return in->nb[k][q]; }
    __host__ __device__ T I_s() const { return in->I_s; }
    __host__ __device__ T tap(int q) const { return in->tap[q]; }
    __host__ __device__ T ybar(int q) const { return yb[q]; }
    __host__ __device__ void out(int q, T v, T) { y[q] = v; }
    __host__ __device__ void add_mu(int q, T v) { xb->mu[q] += v; }
    __host__ __device__ void add_msg(int k, int q, T v) { xb->msg[27 * k + q] += v; }
    __host__ __device__ void add_nm(int q, T v) { xb->nm[q] += v; }
    __host__ __device__ void add_nb(int k, int q, T v) { xb->nb[k][q] += v; }
    __host__ __device__ void add_Is(T v) { xb->I_s += v; }
    __host__ __device__ void add_tap(int q, T v) { xb->tap[q] += v; }
    __host__ __device__ void add_lamD(T v) { xb->lam_D += v; }
    __host__ __device__ void add_isD(T v) { xb->inv_sigma_D += v; }
    __host__ __device__ void add_lamN(T v) { xb->lam_N += v; }
};

// the update's outputs y and, for the output adjoint yb, the input adjoints xb
static void run(const PixIn& in, const PixCtx<T>& c0, const T* yb, PixIn& xb, T* y) {
    PixCtx<T> c = c0;
    c.lam_D = in.lam_D;
    c.inv_sigma_D = in.inv_sigma_D;
    c.lam_N = in.lam_N;
    HostIO io{&in, &xb, yb, y, &c, {}, {}, {}};
    pixel_vjp(io, c);
}

static std::mt19937_64 rng(7);
static double U(double a, double b) { return std::uniform_real_distribution<double>(a, b)(rng); }
static double N01() { return std::normal_distribution<double>(0, 1)(rng); }

// packed symmetric positive definite 6x6 with log-uniform eigenvalues in [lo, hi]
static void rand_spd(double* P, double lo, double hi) {
    double Q[36], A[36];
    for (int i = 0; i < 36; ++i) A[i] = N01();
    for (int c = 0; c < 6; ++c) {  // Gram-Schmidt on the columns
        for (int k = 0; k < c; ++k) {
            double d = 0;
            for (int r = 0; r < 6; ++r) d += A[6 * r + c] * Q[6 * r + k];
            for (int r = 0; r < 6; ++r) A[6 * r + c] -= d * Q[6 * r + k];
        }
        double n = 0;
        for (int r = 0; r < 6; ++r) n += A[6 * r + c] * A[6 * r + c];
        n = std::sqrt(n);
        for (int r = 0; r < 6; ++r) Q[6 * r + c] = A[6 * r + c] / n;
    }
    double ev[6];
    for (int i = 0; i < 6; ++i) ev[i] = std::exp(U(std::log(lo), std::log(hi)));
    for (int r = 0; r < 6; ++r)
        for (int c = 0; c <= r; ++c) {
            double s = 0;
            for (int k = 0; k < 6; ++k) s += Q[6 * r + k] * ev[k] * Q[6 * c + k];
            P[pidx(r, c)] = s;
        }
}

int main(int argc, char** argv) {
    const int huber = argc > 1 ? std::atoi(argv[1]) : 0;
    const int kase = argc > 2 ? std::atoi(argv[2]) : 0;
    // geometry and weights of a 64x48 image at pixel (20, 14); sigma_R = 4e-4
    PixCtx<T> c;
    c.u = 20;
    c.v = 14;
    c.W = 64;
    c.H = 48;
    c.fx = c.fy = 60;
    c.cx = 32;
    c.cy = 24;
    c.ifx = c.ify = 1.0 / 60;
    c.d_prior = 0.3;
    c.lam_P = 400;
    c.lam_Z = 1;
    c.lam_R = 1 / (4e-4 * 4e-4);
    c.beta = 0.5;
    c.t_huber = huber ? 2.0 : 400.0;
    PixIn in;
    std::memset(&in, 0, sizeof(in));
    for (int k = 0; k < 6; ++k) in.mu[k] = 0.01 * N01();
    in.mu[6] = 0.4;
    for (int k = 0; k < 4; ++k) {
        c.has[k] = true;
        c.m[k] = 0.01 * N01();
        rand_spd(in.msg + 27 * k, 1, c.lam_R);
        for (int q = 0; q < 6; ++q) in.msg[27 * k + 21 + q] = N01();
    }
    for (int q = 0; q < 8; ++q) in.nm[q] = q % 2 ? 10 * N01() : U(1, 1e6);
    for (int k = 0; k < 4; ++k) {
        double* nb = in.nb[k];
        for (int q = 0; q < 6; ++q) nb[NB_XJ + q] = in.mu[q] + 1e-4 * N01();
        nb[NB_DJ] = 0.4 + 0.01 * N01();
        double other[21], mine[21];  // M_p,j = the message to this pixel + the rest
        rand_spd(other, 1, c.lam_R);
        rand_spd(mine, 1, c.lam_R);
        for (int q = 0; q < 21; ++q) {
            nb[NB_ML + q] = mine[q];
            nb[NB_MP + q] = mine[q] + other[q];
        }
        for (int q = 0; q < 6; ++q) nb[NB_MP + pidx(q, q)] += c.lam_P;
        for (int q = 0; q < 6; ++q) nb[NB_ME + q] = N01();
        for (int q = 0; q < 6; ++q) nb[NB_U + q] = 300 * N01();
        nb[NB_NN] = U(1, 1e6);
        nb[NB_S] = nb[NB_NN] + U(1, 1e6);
        nb[NB_NE] = 10 * N01();
    }
    in.I_s = huber ? 0.9 : 0.5;  // with huber, |r| / sigma_D well above the threshold
    for (int q = 0; q < 12; ++q) in.tap[q] = q < 4 ? U(0.2, 0.8) : 0.05 * N01();
    in.lam_D = 1 / (5e-3 * 5e-3);
    in.inv_sigma_D = 1 / 5e-3;
    in.lam_N = 1e6;
    // the bilinear cell of the warp at the mean, and the recorded decisions
    {
        T R[9], t[3], Xt[3];
        se3_exp(in.mu, R, t);
        const T z = std::exp(in.mu[6]);
        const T Xs[3] = {z * (c.u - c.cx) * c.ifx, z * (c.v - c.cy) * c.ify, z};
        mat3_vec(R, Xs, Xt);
        for (int i = 0; i < 3; ++i) Xt[i] += t[i];
        c.x0 = (int)std::floor(c.fx * Xt[0] / Xt[2] + c.cx);
        c.y0 = (int)std::floor(c.fy * Xt[1] / Xt[2] + c.cy);
        c.clamp_x = c.clamp_y = false;
        c.br = BR_VALID | (huber ? BR_HUBER : 0) | (kase == 1 ? BR_SKIP : 0);
        if (kase == 2) c.has[0] = c.has[2] = false;
    }
    // a random output adjoint, each plane scaled by the output's magnitude
    std::vector<T> zero(N_OUT, 0.0), yb(N_OUT), y(N_OUT);
    PixIn xb;
    std::memset(&xb, 0, sizeof(xb));
    run(in, c, zero.data(), xb, y.data());
    for (int p = 0; p < N_OUT; ++p) yb[p] = N01() / std::fmax(1.0, std::fabs(y[p]));
    std::memset(&xb, 0, sizeof(xb));
    run(in, c, yb.data(), xb, y.data());
    auto loss = [&](const PixIn& x) {
        PixIn unused;
        std::memset(&unused, 0, sizeof(unused));
        std::vector<T> yy(N_OUT);
        run(x, c, zero.data(), unused, yy.data());
        double L = 0;
        for (int p = 0; p < N_OUT; ++p) L += yb[p] * yy[p];
        return L;
    };
    const int n_in = sizeof(PixIn) / sizeof(T);
    double worst = 0;
    int bad = 0, nz = 0;
    for (int i = 0; i < n_in; ++i) {
        PixIn a = in, b = in;
        const double x0 = reinterpret_cast<const double*>(&in)[i];
        const double h = 1e-6 * std::fmax(1e-3, std::fabs(x0));
        reinterpret_cast<double*>(&a)[i] += h;
        reinterpret_cast<double*>(&b)[i] -= h;
        const double fd = (loss(a) - loss(b)) / (2 * h);
        const double an = reinterpret_cast<const double*>(&xb)[i];
        nz += an != 0.0;
        const double rel = std::fabs(fd - an) / std::fmax(1e-8, std::fmax(std::fabs(fd), std::fabs(an)));
        // an error is counted when it is relatively large and moves L visibly
        const double in_loss = std::fabs(fd - an) * std::fmax(1e-3, std::fabs(x0));
        if (in_loss > 1e-7) {
            if (rel > 1e-4) {
                if (bad < 10) std::printf("input %d: fd %.6e adjoint %.6e rel %.1e\n", i, fd, an, rel);
                bad++;
            }
            if (rel > worst) worst = rel;
        }
    }
    std::printf("inputs %d nonzero %d mismatches %d worst %.2e\n", n_in, nz, bad, worst);
    return 0;
}
