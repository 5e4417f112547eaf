// Kernels of the GB300 direct-coupling multi-level lattice Boltzmann library.
#pragma once

#include <cuda.h>  // CUtensorMap

#include "lbm_device.cuh"

namespace lbmg {

// ------------------------------------------------------------------ interface views
// Interface tables hold values in the arithmetic type R of the storage (double
// for FP64 storage, float for FP32 and FP16-shifted storage); the
// equilibrium/non-equilibrium rescalings of Eqs. (rescff) and (rescfc) are
// evaluated in FP64 in every mode.
struct IfaceDev {
    int nTF, nIE, nRing;
    const int *tf_f;                // [nTF][3] fine-level box coordinates of TF nodes
    const int *tf_c;                // [nTF][3] coarse-level box coordinates
    const unsigned int *tf_kf;      // fine-known populations
    const unsigned int *tf_kc;      // coarse-known populations
    const unsigned int *tf_gc;      // gamma_i = c (Table 1)
    const signed char *tf_rkind;    // [nTF][2D] gradient stencil reference kind
    const int *tf_ridx;             // [nTF][2D] reference: fine node index / TF index / ring index
    const int *ie_f;                // [nIE][3] fine-level box coordinates of hanging nodes
    const unsigned int *ie_kf;
    const int *ie_nst;
    const int *ie_st;               // [nIE][16] TF indices
    const void *ie_w;               // [nIE][16] Lagrange weights in the arithmetic type R
    const int *ring_c;              // [nRing][3] coarse-level box coordinates
    void *hist_f;                   // [3][Q][nTF] coarse post-stream populations at TF nodes (type R)
    void *hist_m;                   // [3][4][nRing] coarse post-stream macros on the ring (type R)
    int tfc_base;                   // table index of the first TF node in the coarse level's table
    double R;                       // Eq. (fneqResc): R = tau_f / (2 tau_c)
    float Rf;                       // R in FP32
    double Rinv;                    // 1 / R
};

struct TimeW {
    int slot[3];   // t - dt^c, t, t + dt^c
    double w[3];   // weights (Eq. TempInt, linear on the first coarse step, [0,0,1] on sync)
    float wf[3];   // the same in FP32
    int nz;        // bit k: w[k] != 0
};

// Eq. (TempInt) weights of the parent's history slots for a fine sub-step: phase 1
// (synchronous) takes the parent's new state, the first coarse step interpolates
// linearly, later ones quadratically through t - dt^c, t, t + dt^c.  kp is the
// parent's step index; the history ring holds slot (kp + 1) % 3 as the newest.
__host__ __device__ __forceinline__ TimeW time_weights(int phase, long long kp)
{
    TimeW tw{};
    tw.slot[0] = (int)((kp + 2) % 3);
    tw.slot[1] = (int)(kp % 3);
    tw.slot[2] = (int)((kp + 1) % 3);
    if (phase == 1) {
        tw.w[0] = 0.0, tw.w[1] = 0.0, tw.w[2] = 1.0;
        tw.wf[0] = 0.0f, tw.wf[1] = 0.0f, tw.wf[2] = 1.0f;
        tw.nz = 4;
    } else if (kp == 0) {
        tw.w[0] = 0.0, tw.w[1] = 0.5, tw.w[2] = 0.5;
        tw.wf[0] = 0.0f, tw.wf[1] = 0.5f, tw.wf[2] = 0.5f;
        tw.nz = 6;
    } else {
        tw.w[0] = -1.0 / 8.0, tw.w[1] = 3.0 / 4.0, tw.w[2] = 3.0 / 8.0;
        tw.wf[0] = -1.0f / 8.0f, tw.wf[1] = 3.0f / 4.0f, tw.wf[2] = 3.0f / 8.0f;
        tw.nz = 7;
    }
    return tw;
}

// weight k of a TimeW in the arithmetic type R
template <typename R> __device__ __forceinline__ R tw_w(const TimeW &tw, int k);
template <> __device__ __forceinline__ double tw_w<double>(const TimeW &tw, int k) { return tw.w[k]; }
template <> __device__ __forceinline__ float tw_w<float>(const TimeW &tw, int k) { return tw.wf[k]; }

__device__ __forceinline__ int box_index(const LevelGeo &g, int x, int y, int z)
{
    return x + g.px * (y + g.n[1] * z);
}

// index of (x,y,z) + (dx,dy,dz) with periodic wrap, -1 off a non-periodic box
__device__ __forceinline__ int nb_index(const LevelGeo &g, int x, int y, int z, int dx, int dy, int dz)
{
    x += dx;
    y += dy;
    z += dz;
    if (!wrap_coord(x, g.n[0], g.per[0]) || !wrap_coord(y, g.n[1], g.per[1]) || !wrap_coord(z, g.n[2], g.per[2]))
        return -1;
    return box_index(g, x, y, z);
}

// post-stream moments of a node whose Q sources are all nodes of the level (pull)
template <int Q, typename S>
__device__ __forceinline__ void pulled_moments(const LevelGeo &g, const S *__restrict__ f, int x, int y, int z,
                                               typename St<S>::R &rho, typename St<S>::R *u)
{
    using L = Lat<Q>;
    using R = typename St<S>::R;
    constexpr int D = L::D;
    R r = R(0), m[3] = {R(0), R(0), R(0)};
#pragma unroll
    for (int i = 0; i < Q; i++) {
        const int s = nb_index(g, x, y, z, -L::c(i, 0), -L::c(i, 1), -L::c(i, 2));
        const R v = s >= 0 ? St<S>::ld(f, (long long)i * g.pitch + s, g.shift[i]) : R(0);
        r += v;
#pragma unroll
        for (int a = 0; a < D; a++)
            if (L::c(i, a) != 0) m[a] += R(L::c(i, a)) * v;
    }
    rho = r;
#pragma unroll
    for (int a = 0; a < 3; a++) u[a] = a < D ? m[a] / r : R(0);
}

// storage shift of a run-time population index (FP16-shifted storage; compile-time
// indices into the shift table, no local copy of the kernel parameter)
template <int Q>
__device__ __forceinline__ float lane_shift(const LevelGeo &g, int i)
{
    float s = 0.0f;
#pragma unroll
    for (int j = 0; j < Q; j++)
        if (i == j) s = g.shift[j];
    return s;
}

// ------------------------------------------------------------------ interface nodes, W-lane segments
// Small interfaces: one 16- (D2Q9) or 32-lane (D3Q19) segment per node, one population
// per lane, warp-shuffle sums: many threads per node keep the latency of a launch that
// has few nodes short.  (Large interfaces use the one-node-per-thread bodies below.)

// ------------------------------------------------------------------ TF reconstruction
// segmented warp reduction over the W lanes that hold one TF node's populations
template <int W, typename T>
__device__ __forceinline__ T seg_sum(T v)
{
#pragma unroll
    for (int o = W / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o, W);
    return v;
}

// velocity and weight of a run-time population index
template <int Q, typename T>
__device__ __forceinline__ void lane_lattice(int i, int &cx, int &cy, int &cz, T &w)
{
    using L = Lat<Q>;
    cx = cy = cz = 0;
    w = T(0);
#pragma unroll
    for (int j = 0; j < Q; j++)
        if (i == j) {
            cx = L::c(j, 0);
            cy = L::c(j, 1);
            cz = L::c(j, 2);
            w = T(L::w(j));
        }
}

// Eq. (fEq_herm) for one population and its derivatives with respect to (rho, u)
template <int D, typename T>
__device__ __forceinline__ T feq_lane(const int *c, T w, T rho, const T *u, T *d)
{
    const T third = T(1) / T(3);
    T cu = T(0), uu = T(0), h3 = T(0);
#pragma unroll
    for (int a = 0; a < D; a++) {
        cu += T(c[a]) * u[a];
        uu += u[a] * u[a];
    }
    T dh3[3] = {T(0), T(0), T(0)};
#pragma unroll
    for (int a = 0; a < D; a++)
#pragma unroll
        for (int b = 0; b < D; b++)
            if (a != b) {
                const T k = (T(c[a] * c[a]) - third) * T(c[b]);
                h3 += k * u[a] * u[a] * u[b];
                dh3[a] += k * T(2) * u[a] * u[b];
                dh3[b] += k * u[a] * u[a];
            }
    const T p = T(1) + T(3) * cu + T(4.5) * cu * cu - T(1.5) * uu + T(13.5) * h3;
    if (d) {
        d[0] = w * p;
#pragma unroll
        for (int g = 0; g < D; g++)
            d[1 + g] = w * rho * (T(3) * T(c[g]) + T(9) * cu * T(c[g]) - T(3) * u[g] + T(13.5) * dh3[g]);
    }
    return w * rho * p;
}

// Eq. (fEq_herm) of one population in FP64, for the rescalings of Eqs. (rescff) and
// (rescfc), written with few FP64 operations (GB300 runs FP64 at 1/64 of the FP32
// rate).  For velocities with components in {-1, 0, 1}, with cu = c.u, uu = u.u,
// V = sum_a c_a^2 u_a^2 and W3 = sum_b c_b u_b^3, the third-order Hermite term
// sum_{a != b} (c_a^2 - 1/3) c_b u_a^2 u_b equals cu (V - uu/3) - (2/3) W3: the inner
// sum over a != b of (c_a^2 - 1/3) u_a^2 is V - uu/3 - (2/3) u_b^2 when c_b^2 = 1.
template <int D>
__device__ __forceinline__ double feq_rescale(const int *c, double w, double rho, const double *u)
{
    double u2[3], cu = 0.0, uu = 0.0, V = 0.0, W3 = 0.0;
#pragma unroll
    for (int a = 0; a < D; a++) {
        u2[a] = u[a] * u[a];
        uu += u2[a];
        const double s = c[a] > 0 ? u[a] : (c[a] < 0 ? -u[a] : 0.0);  // c_a u_a
        cu += s;
        V += c[a] != 0 ? u2[a] : 0.0;
        W3 += s * u2[a];
    }
    const double h3 = cu * (V - uu * (1.0 / 3.0)) - (2.0 / 3.0) * W3;
    const double p = 1.0 + cu * (3.0 + 4.5 * cu) - 1.5 * uu + 13.5 * h3;
    return (w * rho) * p;
}

// Newton-Raphson for F(X) = sum_i Gamma_i Phi_i (fhat_i - f0_i(X)) = 0 (Eq. system_fi)
// with one population per lane of a W-lane segment; started from the plain moments
// of fhat and stopped once max|dX| < tol (Eq. updated_macro).  Every lane of a
// segment holds the same X.  All 32 lanes of the warp run the same number of
// iterations (the shuffles need the full warp): a segment that has converged, or
// is inactive, keeps its X while the others finish.  Returns the iteration count
// at convergence, or -1 (singular Jacobian or no convergence in 10 iterations).
template <int Q, int W, typename T>
__device__ int newton_seg(const int *c, T w, T fhat, T gam, T tol, bool active, T *X)
{
    constexpr int D = Lat<Q>::D, n = D + 1;
    T phi[4] = {T(1), T(c[0]), T(c[1]), T(c[2])};
    T s[4];
#pragma unroll
    for (int r = 0; r < n; r++) s[r] = seg_sum<W>(phi[r] * fhat);
    X[0] = s[0];
#pragma unroll
    for (int a = 0; a < D; a++) X[1 + a] = s[1 + a] / s[0];
    int done = active ? 0 : 11;  // iteration of convergence; 11 = inactive
    bool bad = false;
    for (int it = 1; it <= 10; it++) {
        T d[4];
        const T fe = feq_lane<D, T>(c, w, X[0], X + 1, d);
        T F[4], J[16];
#pragma unroll
        for (int r = 0; r < n; r++) {
            F[r] = seg_sum<W>(gam * phi[r] * (fhat - fe));
#pragma unroll
            for (int k = 0; k < n; k++) J[r * n + k] = seg_sum<W>(-gam * phi[r] * d[k]);
        }
        // Gaussian elimination with partial pivoting on J dX = -F (same on every lane)
        T b[4], dX[4];
        bool sing = false;
#pragma unroll
        for (int r = 0; r < n; r++) b[r] = -F[r];
#pragma unroll
        for (int k = 0; k < n; k++) {
            int p = k;
#pragma unroll
            for (int r = k + 1; r < n; r++)
                if (fabs(J[r * n + k]) > fabs(J[p * n + k])) p = r;
#pragma unroll
            for (int r = k + 1; r < n; r++)
                if (r == p) {
#pragma unroll
                    for (int c2 = 0; c2 < n; c2++) {
                        const T t0 = J[k * n + c2];
                        J[k * n + c2] = J[r * n + c2];
                        J[r * n + c2] = t0;
                    }
                    const T t1 = b[k];
                    b[k] = b[r];
                    b[r] = t1;
                }
            if (J[k * n + k] == T(0)) {
                sing = true;
                J[k * n + k] = T(1);
            }
#pragma unroll
            for (int r = k + 1; r < n; r++) {
                const T m = J[r * n + k] / J[k * n + k];
#pragma unroll
                for (int c2 = k; c2 < n; c2++) J[r * n + c2] -= m * J[k * n + c2];
                b[r] -= m * b[k];
            }
        }
#pragma unroll
        for (int k = n - 1; k >= 0; k--) {
            T sum = b[k];
#pragma unroll
            for (int c2 = k + 1; c2 < n; c2++) sum -= J[k * n + c2] * dX[c2];
            dX[k] = sum / J[k * n + k];
        }
        if (done == 0) {
            if (sing) {
                bad = true;
                done = 11;
            } else {
                T mx = T(0);
#pragma unroll
                for (int r = 0; r < n; r++) {
                    X[r] += dX[r];
                    mx = fmax(mx, fabs(dX[r]));
                }
                if (mx < tol) done = it;
            }
        }
        if (!__any_sync(0xffffffffu, done == 0)) break;
    }
    return (bad || done == 0 || done == 11) ? -1 : done;
}

// Newton at TF nodes (Eq. system_fi) in the storage's arithmetic type, then, in FP64,
// the fine rebuild of gamma=c populations (Eq. rescff) and on sync sub-steps the
// coarse rebuild of all populations (Eq. rescfc).  One W-lane segment per TF node.
template <int Q, typename S>
__device__ __forceinline__ void recon_seg(int bid, IfaceDev I, LevelDev F, LevelDev Cl, const S *__restrict__ ff,
                                                 TimeW tw, int sync, int *status, int *max_iters)
{
    using L = Lat<Q>;
    using R = typename St<S>::R;
    constexpr int D = L::D;
    constexpr int W = Q <= 16 ? 16 : 32;
    const int lane = threadIdx.x & 31;
    const int seg = (bid * blockDim.x + threadIdx.x) / W;
    const int i = lane % W;
    const bool live = seg < I.nTF;
    const int t = live ? seg : 0;
    int c[3];
    R wd;
    lane_lattice<Q>(i, c[0], c[1], c[2], wd);
    const bool pop = live && i < Q;
    // lanes beyond Q carry nothing; a segment past the last TF node solves the rest state
    R fhat = (!live && i < Q) ? wd : R(0), gam = (!live && i < Q) ? R(1) : R(0);
    const unsigned int gcm = I.tf_gc[t];
    if (pop) {
        if ((gcm >> i) & 1u) {
            const R *hf = (const R *)I.hist_f;
            R s = R(0);
#pragma unroll
            for (int k = 0; k < 3; k++)
                if ((tw.nz >> k) & 1) s += tw_w<R>(tw, k) * hf[((long long)tw.slot[k] * Q + i) * I.nTF + t];
            fhat = s;
            gam = sizeof(R) == 8 ? (R)I.R : (R)I.Rf;
        } else {
            if ((I.tf_kf[t] >> i) & 1u) {
                const int s = nb_index(F.g, I.tf_f[3 * t], I.tf_f[3 * t + 1], I.tf_f[3 * t + 2], -c[0], -c[1], -c[2]);
                if (s >= 0) fhat = St<S>::ld(ff, (long long)i * F.g.pitch + s, lane_shift<Q>(F.g, i));
            }
            gam = R(1);
        }
    }
    R X[4] = {R(0), R(0), R(0), R(0)};
    const R tol = sizeof(R) == 8 ? R(1e-12) : R(2e-6);
    const int it = newton_seg<Q, W, R>(c, i < Q ? wd : R(0), fhat, gam, tol, live, X);
    if (!live) return;
    if (it < 0) {
        if (i == 0) atomicOr(status, ST_NEWTON);
        return;
    }
    if (i == 0) atomicMax(max_iters, it);
    R *fpop = (R *)F.if_pop;
    R *fmac = (R *)F.if_mac;
    if (i < Q) {
        // FP64 equilibrium / non-equilibrium rescaling
        double w64;
        int cc[3];
        lane_lattice<Q>(i, cc[0], cc[1], cc[2], w64);
        const double Xd[3] = {(double)X[1], (double)X[2], (double)X[3]};
        const double fe = feq_rescale<D>(c, w64, (double)X[0], Xd);
        const double fh = (double)fhat;
        const double v = ((gcm >> i) & 1u) ? fe + I.R * (fh - fe) : fh;
        fpop[(long long)i * F.nif + t] = (R)v;
        if (sync) ((R *)Cl.if_pop)[(long long)i * Cl.nif + I.tfc_base + t] = (R)(fe + (v - fe) * I.Rinv);
    }
    if (i < 4) {
        const R xv = i <= D ? X[i] : R(0);
        fmac[(long long)i * F.nif + t] = xv;
        if (sync) ((R *)Cl.if_mac)[(long long)i * Cl.nif + I.tfc_base + t] = xv;
    }
}

// ------------------------------------------------------------------ history push
// post-stream coarse populations at TF nodes (coarse-known ones) and post-stream
// macros at ring nodes, for the child level's Eq. (TempInt).  One W-lane segment
// per node, lane i handles population i (TF segments first, then ring segments).
template <int Q, typename S>
__device__ __forceinline__ void hist_seg(int bid, IfaceDev I, LevelGeo gc, const S *__restrict__ fc, int slot, int seed)
{
    using L = Lat<Q>;
    using R = typename St<S>::R;
    constexpr int D = L::D;
    constexpr int W = Q <= 16 ? 16 : 32;
    const int seg = (bid * blockDim.x + threadIdx.x) / W;
    const int i = threadIdx.x % W;
    int c[3];
    R wd;
    lane_lattice<Q>(i, c[0], c[1], c[2], wd);
    const bool is_tf = seg < I.nTF;
    const int r = seg - I.nTF;
    const bool live_ring = !is_tf && r < I.nRing;
    if (is_tf && i < Q) {
        const int t = seg;
        const int x = I.tf_c[3 * t], y = I.tf_c[3 * t + 1], z = I.tf_c[3 * t + 2];
        // seed: slot 0 holds the initial state itself; otherwise the post-stream value
        const int s = seed ? box_index(gc, x, y, z)
                           : (((I.tf_kc[t] >> i) & 1u) ? nb_index(gc, x, y, z, -c[0], -c[1], -c[2]) : -1);
        ((R *)I.hist_f)[((long long)slot * Q + i) * I.nTF + t] =
            s >= 0 ? St<S>::ld(fc, (long long)i * gc.pitch + s, lane_shift<Q>(gc, i)) : R(0);
    }
    R v = R(0);
    if (live_ring && i < Q) {
        const int x = I.ring_c[3 * r], y = I.ring_c[3 * r + 1], z = I.ring_c[3 * r + 2];
        const int s = seed ? box_index(gc, x, y, z) : nb_index(gc, x, y, z, -c[0], -c[1], -c[2]);
        if (s >= 0) v = St<S>::ld(fc, (long long)i * gc.pitch + s, lane_shift<Q>(gc, i));
    }
    const R rho = seg_sum<W>(v);
    R m[3] = {R(0), R(0), R(0)};
#pragma unroll
    for (int a = 0; a < D; a++) m[a] = seg_sum<W>(R(c[a]) * v);
    if (live_ring && i < 4) {
        R *h = (R *)I.hist_m + (long long)slot * 4 * I.nRing;
        h[(long long)i * I.nRing + r] = i == 0 ? rho : (i <= D ? m[i - 1] / rho : R(0));
    }
}

// ------------------------------------------------------------------ TF gradients
// Sec. 3.3: centred differences over the coarse stencil (fine nodes two fine cells
// inward, TF neighbours along the interface with their X, coarse ring nodes outward,
// time-interpolated on async sub-steps), rescaled by 1/2 for the fine level.  One
// W-lane segment per TF node: the lanes pull the populations of fine neighbours in
// parallel; every lane then holds the stencil and lanes 0..11 write S and C.
template <int Q, typename S>
__device__ __forceinline__ void grad_seg(int bid, IfaceDev I, LevelDev F, LevelDev Cl, const S *__restrict__ ff,
                                                TimeW tw, int sync)
{
    using L = Lat<Q>;
    using R = typename St<S>::R;
    constexpr int D = L::D;
    constexpr int W = Q <= 16 ? 16 : 32;
    const int seg = (bid * blockDim.x + threadIdx.x) / W;
    const int i = threadIdx.x % W;
    const bool live = seg < I.nTF;
    const int t = live ? seg : 0;
    int c[3];
    R wd;
    lane_lattice<Q>(i, c[0], c[1], c[2], wd);
    const R *fmac = (const R *)F.if_mac;
    const R *hm = (const R *)I.hist_m;
    // all stencil references first, then every load of every reference, then the
    // reductions: two rounds of dependent loads instead of two per stencil point
    signed char kind[3][2];
    int ref[3][2];
#pragma unroll
    for (int b = 0; b < D; b++)
#pragma unroll
        for (int s = 0; s < 2; s++) {
            const int k = t * 2 * D + 2 * b + s;
            kind[b][s] = I.tf_rkind[k];
            ref[b][s] = I.tf_ridx[k];
        }
    R v[3][2], rho[3][2], u[3][2][3];
#pragma unroll
    for (int b = 0; b < D; b++)
#pragma unroll
        for (int s = 0; s < 2; s++) {
            const int kd = kind[b][s], rf = ref[b][s];
            // fine neighbour: lane i pulls its population i (zero for other kinds)
            v[b][s] = R(0);
            if (live && kd == RK_FINE && i < Q) {
                const int x = rf % F.g.n[0], yz = rf / F.g.n[0];
                const int src = nb_index(F.g, x, yz % F.g.n[1], yz / F.g.n[1], -c[0], -c[1], -c[2]);
                if (src >= 0) v[b][s] = St<S>::ld(ff, (long long)i * F.g.pitch + src, lane_shift<Q>(F.g, i));
            }
            rho[b][s] = R(0);
#pragma unroll
            for (int a = 0; a < 3; a++) u[b][s][a] = R(0);
            if (kd == RK_TF) {
                rho[b][s] = fmac[rf];
#pragma unroll
                for (int a = 0; a < D; a++) u[b][s][a] = fmac[(long long)(1 + a) * F.nif + rf];
            } else if (kd != RK_FINE) {
#pragma unroll
                for (int j = 0; j < 3; j++) {
                    if (!((tw.nz >> j) & 1)) continue;
                    const R *h = hm + (long long)tw.slot[j] * 4 * I.nRing;
                    const R wj = tw_w<R>(tw, j);
                    rho[b][s] += wj * h[rf];
#pragma unroll
                    for (int a = 0; a < D; a++) u[b][s][a] += wj * h[(long long)(1 + a) * I.nRing + rf];
                }
            }
        }
#pragma unroll
    for (int b = 0; b < D; b++)
#pragma unroll
        for (int s = 0; s < 2; s++) {
            const R r = seg_sum<W>(v[b][s]);
            R uu[3];
#pragma unroll
            for (int a = 0; a < D; a++) uu[a] = seg_sum<W>(R(c[a]) * v[b][s]);
            if (kind[b][s] == RK_FINE) {
                rho[b][s] = r;
#pragma unroll
                for (int a = 0; a < D; a++) u[b][s][a] = uu[a] / r;
            }
        }
    if (!live) return;
    R Sg[6], Cg[6];
    fd_gradients<D, R>(rho, u, R(0.5), Sg, Cg);  // coarse units: neighbours one coarse cell away
    if (i < 12) {
        const int k = i % 6;
        R *dstF = (R *)(i < 6 ? F.if_S : F.if_C);
        const R val = i < 6 ? Sg[k] : Cg[k];
        dstF[(long long)k * F.nif + t] = R(0.5) * val;
        if (sync) ((R *)(i < 6 ? Cl.if_S : Cl.if_C))[(long long)k * Cl.nif + I.tfc_base + t] = val;
    }
}

// ------------------------------------------------------------------ hanging nodes
// 4-point 1-D Lagrange along the interface (tensor order over odd axes, one-sided
// next to corners) of missing populations; macros are the moments.  One W-lane
// segment per hanging node, lane i completes population i.  S and C of hanging
// nodes are interpolated with the same stencil by the 2-D tile kernel where they are
// used (collide_store) and for D3Q19 by k_ie_sc after this launch.

// stencil slots a hanging node may use (rows of [n_ie][16]): 4 points along its odd
// axis in 2-D, a 4 x 4 tensor over its two odd in-face axes in 3-D
template <int D>
constexpr int kIeSlots = D == 2 ? 4 : 16;

template <int Q, typename S>
__device__ __forceinline__ void ie_seg(int bid, IfaceDev I, LevelDev F, const S *__restrict__ ff)
{
    using L = Lat<Q>;
    using R = typename St<S>::R;
    constexpr int D = L::D;
    constexpr int W = Q <= 16 ? 16 : 32;
    const int seg = (bid * blockDim.x + threadIdx.x) / W;
    const int i = threadIdx.x % W;
    const bool live = seg < I.nIE;
    const int e = live ? seg : 0;
    int c[3];
    R wd;
    lane_lattice<Q>(i, c[0], c[1], c[2], wd);
    const int nif = F.nif;
    const int row = I.nTF + e;  // table index of this hanging node
    R *fpop = (R *)F.if_pop;
    const int nst = I.ie_nst[e];
    R v = R(0);
    if (live && i < Q) {
        if ((I.ie_kf[e] >> i) & 1u) {
            const int s = nb_index(F.g, I.ie_f[3 * e], I.ie_f[3 * e + 1], I.ie_f[3 * e + 2], -c[0], -c[1], -c[2]);
            if (s >= 0) v = St<S>::ld(ff, (long long)i * F.g.pitch + s, lane_shift<Q>(F.g, i));
        } else {
            // every stencil slot read at once, then the used TF rows at once
            constexpr int NS = kIeSlots<D>;
            const R *iw = (const R *)I.ie_w;
            int st[NS];
            R w[NS];
#pragma unroll
            for (int k = 0; k < NS; k++) {
                st[k] = I.ie_st[e * 16 + k];
                w[k] = iw[e * 16 + k];
            }
#pragma unroll
            for (int k = 0; k < NS; k++)
                if (k < nst) v += w[k] * fpop[(long long)i * nif + st[k]];
        }
        fpop[(long long)i * nif + row] = v;
    }
    const R rho = seg_sum<W>(v);
    R m[3] = {R(0), R(0), R(0)};
#pragma unroll
    for (int a = 0; a < D; a++) m[a] = seg_sum<W>(R(c[a]) * v);
    if (live && i < 4) ((R *)F.if_mac)[(long long)i * nif + row] = i == 0 ? rho : (i <= D ? m[i - 1] / rho : R(0));
}


// ------------------------------------------------------------------ interface nodes, one per thread
// Large interfaces take one node per thread.  A node's populations are a
// compile-time loop (every lattice constant is a constant expression), the sums over
// populations are register sums, and neighbouring threads hold neighbouring nodes of
// an interface (the node lists are in box order), so the loads of one population by a
// warp fall in few sectors.

// Eq. (fEq_herm) of population I at X = (rho, u) and, if d is not null, its
// derivatives with respect to (rho, u_1 .. u_D)
template <int Q, int I, typename T>
__device__ __forceinline__ T feq_pop(T rho, const T *u, T *d)
{
    using L = Lat<Q>;
    constexpr int D = L::D;
    const T w = T(L::w(I));
    T cu = T(0), uu = T(0), h3 = T(0), dh3[3] = {T(0), T(0), T(0)};
    static_for<D>([&](auto ac) {
        constexpr int a = decltype(ac)::value;
        if constexpr (L::c(I, a) > 0) cu += u[a];
        else if constexpr (L::c(I, a) < 0) cu -= u[a];
        uu += u[a] * u[a];
    });
    static_for<D>([&](auto ac) {
        constexpr int a = decltype(ac)::value;
        static_for<D>([&](auto bc) {
            constexpr int b = decltype(bc)::value;
            constexpr int ca = L::c(I, a), cb = L::c(I, b);
            if constexpr (a != b && cb != 0) {
                // H3_aab = (c_a^2 - cs2) c_b
                const T k = T(((double)(ca * ca) - 1.0 / 3.0) * cb);
                h3 += k * u[a] * u[a] * u[b];
                if (d) {
                    dh3[a] += k * T(2) * u[a] * u[b];
                    dh3[b] += k * u[a] * u[a];
                }
            }
        });
    });
    const T p = T(1) + T(3) * cu + T(4.5) * cu * cu - T(1.5) * uu + T(13.5) * h3;
    if (d) {
        d[0] = w * p;
        static_for<D>([&](auto gc) {
            constexpr int g = decltype(gc)::value;
            constexpr T cg = T(L::c(I, g));
            d[1 + g] = w * rho * (T(3) * cg + T(9) * cu * cg - T(3) * u[g] + T(13.5) * dh3[g]);
        });
    }
    return w * rho * p;
}

// Eq. (fEq_herm) of population I in FP64, for the rescalings of Eqs. (rescff) and
// (rescfc), with the node's velocity terms computed once (GB300 runs FP64 at 1/64 of
// the FP32 rate).  For velocities with components in {-1, 0, 1}, with cu = c.u,
// uu = u.u, V = sum_a c_a^2 u_a^2 and W3 = sum_b c_b u_b^3, the third-order Hermite
// term sum_{a != b} (c_a^2 - 1/3) c_b u_a^2 u_b equals cu (V - uu/3) - (2/3) W3: the
// inner sum over a != b of (c_a^2 - 1/3) u_a^2 is V - uu/3 - (2/3) u_b^2 when c_b^2 = 1.
struct Feq64 {
    double rho, u[3], u2[3], u3[3], uu;
};
template <int D>
__device__ __forceinline__ Feq64 feq64_node(double rho, const double *u)
{
    Feq64 n;
    n.rho = rho;
    n.uu = 0.0;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        n.u[a] = a < D ? u[a] : 0.0;
        n.u2[a] = n.u[a] * n.u[a];
        n.u3[a] = n.u2[a] * n.u[a];
        if (a < D) n.uu += n.u2[a];
    }
    return n;
}
template <int Q, int I>
__device__ __forceinline__ double feq64_pop(const Feq64 &n)
{
    using L = Lat<Q>;
    constexpr int D = L::D;
    double cu = 0.0, V = 0.0, W3 = 0.0;
    static_for<D>([&](auto ac) {
        constexpr int a = decltype(ac)::value;
        if constexpr (L::c(I, a) > 0) {
            cu += n.u[a];
            W3 += n.u3[a];
        } else if constexpr (L::c(I, a) < 0) {
            cu -= n.u[a];
            W3 -= n.u3[a];
        }
        if constexpr (L::c(I, a) != 0) V += n.u2[a];
    });
    const double h3 = cu * (V - n.uu * (1.0 / 3.0)) - (2.0 / 3.0) * W3;
    const double p = 1.0 + cu * (3.0 + 4.5 * cu) - 1.5 * n.uu + 13.5 * h3;
    return (L::w(I) * n.rho) * p;
}

// Newton-Raphson for F(X) = sum_i Gamma_i Phi_i (fhat_i - f0_i(X)) = 0 (Eq. system_fi)
// at one node, Phi = (1, c_i), Gamma_i = gc where bit i of gmask is set (gamma_i = c)
// and 1 otherwise; started from the plain moments of fhat and stopped once
// max|dX| < tol (Eq. updated_macro).  Returns the iteration count at convergence, or
// -1 (singular Jacobian or no convergence in 10 iterations).
template <int Q, typename T>
__device__ int newton_node(const T (&fhat)[Q], unsigned gmask, T gc, T tol, T (&X)[4])
{
    using L = Lat<Q>;
    constexpr int D = L::D, n = D + 1;
    T s0 = T(0), s[3] = {T(0), T(0), T(0)};
    static_for<Q>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        s0 += fhat[i];
        static_for<D>([&](auto ac) {
            constexpr int a = decltype(ac)::value;
            if constexpr (L::c(i, a) > 0) s[a] += fhat[i];
            else if constexpr (L::c(i, a) < 0) s[a] -= fhat[i];
        });
    });
    X[0] = s0;
    X[3] = T(0);
#pragma unroll
    for (int a = 0; a < D; a++) X[1 + a] = s[a] / s0;
    for (int it = 1; it <= 10; it++) {
        T F[4] = {T(0), T(0), T(0), T(0)}, J[16];
#pragma unroll
        for (int k = 0; k < 16; k++) J[k] = T(0);
        static_for<Q>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            T d[4];
            const T fe = feq_pop<Q, i, T>(X[0], X + 1, d);
            const T gam = ((gmask >> i) & 1u) ? gc : T(1);
            const T r = gam * (fhat[i] - fe);
            F[0] += r;
#pragma unroll
            for (int k = 0; k < n; k++) J[k] -= gam * d[k];
            static_for<D>([&](auto ac) {
                constexpr int a = decltype(ac)::value;
                if constexpr (L::c(i, a) != 0) {
                    constexpr T ca = T(L::c(i, a));
                    F[1 + a] += ca * r;
#pragma unroll
                    for (int k = 0; k < n; k++) J[(1 + a) * n + k] -= ca * gam * d[k];
                }
            });
        });
        // Gaussian elimination with partial pivoting on J dX = -F
        T b[4], dX[4];
#pragma unroll
        for (int r = 0; r < n; r++) b[r] = -F[r];
#pragma unroll
        for (int k = 0; k < n; k++) {
            int p = k;
#pragma unroll
            for (int r = k + 1; r < n; r++)
                if (fabs(J[r * n + k]) > fabs(J[p * n + k])) p = r;
#pragma unroll
            for (int r = k + 1; r < n; r++)
                if (r == p) {
#pragma unroll
                    for (int c2 = 0; c2 < n; c2++) {
                        const T t0 = J[k * n + c2];
                        J[k * n + c2] = J[r * n + c2];
                        J[r * n + c2] = t0;
                    }
                    const T t1 = b[k];
                    b[k] = b[r];
                    b[r] = t1;
                }
            if (J[k * n + k] == T(0)) return -1;
#pragma unroll
            for (int r = k + 1; r < n; r++) {
                const T m = J[r * n + k] / J[k * n + k];
#pragma unroll
                for (int c2 = k; c2 < n; c2++) J[r * n + c2] -= m * J[k * n + c2];
                b[r] -= m * b[k];
            }
        }
        T mx = T(0);
#pragma unroll
        for (int k = n - 1; k >= 0; k--) {
            T sum = b[k];
#pragma unroll
            for (int c2 = k + 1; c2 < n; c2++) sum -= J[k * n + c2] * dX[c2];
            dX[k] = sum / J[k * n + k];
        }
#pragma unroll
        for (int r = 0; r < n; r++) {
            X[r] += dX[r];
            mx = fmax(mx, fabs(dX[r]));
        }
        if (mx < tol) return it;
    }
    return -1;
}

// ------------------------------------------------------------------ TF reconstruction
// Newton at TF nodes (Eq. system_fi) in the storage's arithmetic type, then, in FP64,
// the fine rebuild of gamma=c populations (Eq. rescff) and on sync sub-steps the
// coarse rebuild of all populations (Eq. rescfc).  One TF node per thread.
template <int Q, typename S>
__device__ __forceinline__ void recon_node(int bid, IfaceDev I, LevelDev F, LevelDev Cl, const S *__restrict__ ff,
                                           TimeW tw, int sync, int *status, int *max_iters)
{
    using L = Lat<Q>;
    using R = typename St<S>::R;
    constexpr int D = L::D;
    const int t = bid * blockDim.x + threadIdx.x;
    if (t >= I.nTF) return;
    const unsigned gcm = I.tf_gc[t], kfm = I.tf_kf[t];
    const int x = I.tf_f[3 * t], y = I.tf_f[3 * t + 1], z = I.tf_f[3 * t + 2];
    const R *hf = (const R *)I.hist_f;
    R fhat[Q];
    static_for<Q>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        R v = R(0);
        if ((gcm >> i) & 1u) {
#pragma unroll
            for (int k = 0; k < 3; k++)
                if ((tw.nz >> k) & 1) v += tw_w<R>(tw, k) * hf[((long long)tw.slot[k] * Q + i) * I.nTF + t];
        } else if ((kfm >> i) & 1u) {
            const int s = nb_index(F.g, x, y, z, -L::c(i, 0), -L::c(i, 1), -L::c(i, 2));
            if (s >= 0) v = St<S>::ld(ff, (long long)i * F.g.pitch + s, F.g.shift[i]);
        }
        fhat[i] = v;
    });
    R X[4];
    const R tol = sizeof(R) == 8 ? R(1e-12) : R(2e-6);
    const R gc = sizeof(R) == 8 ? (R)I.R : (R)I.Rf;
    const int it = newton_node<Q, R>(fhat, gcm, gc, tol, X);
    if (it < 0) {
        atomicOr(status, ST_NEWTON);
        return;
    }
    {
        const unsigned m = __activemask();
        const int wmax = __reduce_max_sync(m, it);
        if ((int)(threadIdx.x & 31) == __ffs(m) - 1) atomicMax(max_iters, wmax);
    }
    R *fpop = (R *)F.if_pop;
    R *cpop = (R *)Cl.if_pop;
    const double Xd[3] = {(double)X[1], (double)X[2], (double)X[3]};
    const Feq64 nd = feq64_node<D>((double)X[0], Xd);
    static_for<Q>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        // FP64 equilibrium / non-equilibrium rescaling; the equilibrium only where a
        // rescaling uses it (gamma_i = c, or every population of a sync sub-step)
        const bool gc_i = (gcm >> i) & 1u;
        const double fh = (double)fhat[i];
        double v = fh;
        if (gc_i || sync) {
            const double fe = feq64_pop<Q, i>(nd);
            if (gc_i) v = fe + I.R * (fh - fe);
            if (sync) cpop[(long long)i * Cl.nif + I.tfc_base + t] = (R)(fe + (v - fe) * I.Rinv);
        }
        fpop[(long long)i * F.nif + t] = (R)v;
    });
    R *fmac = (R *)F.if_mac;
#pragma unroll
    for (int a = 0; a < 4; a++) {
        const R xv = a <= D ? X[a] : R(0);
        fmac[(long long)a * F.nif + t] = xv;
        if (sync) ((R *)Cl.if_mac)[(long long)a * Cl.nif + I.tfc_base + t] = xv;
    }
}

// ------------------------------------------------------------------ history push
// post-stream coarse populations at TF nodes (coarse-known ones) and post-stream
// macros at ring nodes, for the child level's Eq. (TempInt).  One node per thread:
// items [0, nTF) are TF nodes, [nTF, nTF + nRing) ring nodes.  seed = 1 stores the
// state itself (slot 0 holds the initial state).
template <int Q, typename S>
__device__ __forceinline__ void hist_node(int bid, IfaceDev I, LevelGeo gc, const S *__restrict__ fc, int slot, int seed)
{
    using L = Lat<Q>;
    using R = typename St<S>::R;
    constexpr int D = L::D;
    const int item = bid * blockDim.x + threadIdx.x;
    if (item < I.nTF) {
        const int t = item;
        const int x = I.tf_c[3 * t], y = I.tf_c[3 * t + 1], z = I.tf_c[3 * t + 2];
        const unsigned kcm = I.tf_kc[t];
        R *hf = (R *)I.hist_f;
        static_for<Q>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            const int s = seed ? box_index(gc, x, y, z)
                               : (((kcm >> i) & 1u) ? nb_index(gc, x, y, z, -L::c(i, 0), -L::c(i, 1), -L::c(i, 2)) : -1);
            hf[((long long)slot * Q + i) * I.nTF + t] = s >= 0 ? St<S>::ld(fc, (long long)i * gc.pitch + s, gc.shift[i]) : R(0);
        });
    } else if (item < I.nTF + I.nRing) {
        const int r = item - I.nTF;
        const int x = I.ring_c[3 * r], y = I.ring_c[3 * r + 1], z = I.ring_c[3 * r + 2];
        R rho = R(0), m[3] = {R(0), R(0), R(0)};
        static_for<Q>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            const int s = seed ? box_index(gc, x, y, z) : nb_index(gc, x, y, z, -L::c(i, 0), -L::c(i, 1), -L::c(i, 2));
            const R v = s >= 0 ? St<S>::ld(fc, (long long)i * gc.pitch + s, gc.shift[i]) : R(0);
            rho += v;
            static_for<D>([&](auto ac) {
                constexpr int a = decltype(ac)::value;
                if constexpr (L::c(i, a) > 0) m[a] += v;
                else if constexpr (L::c(i, a) < 0) m[a] -= v;
            });
        });
        R *h = (R *)I.hist_m + (long long)slot * 4 * I.nRing;
        h[r] = rho;
#pragma unroll
        for (int a = 0; a < 3; a++) h[(long long)(1 + a) * I.nRing + r] = a < D ? m[a] / rho : R(0);
    }
}

// ------------------------------------------------------------------ TF gradients
// Sec. 3.3: centred differences over the coarse stencil (fine nodes two fine cells
// inward, TF neighbours along the interface with their X, coarse ring nodes outward,
// time-interpolated on async sub-steps), rescaled by 1/2 for the fine level.  One TF
// node per thread; all stencil references are loaded before any of their data.
template <int Q, typename S>
__device__ __forceinline__ void grad_node(int bid, IfaceDev I, LevelDev F, LevelDev Cl, const S *__restrict__ ff,
                                          TimeW tw, int sync)
{
    using L = Lat<Q>;
    using R = typename St<S>::R;
    constexpr int D = L::D;
    const int t = bid * blockDim.x + threadIdx.x;
    if (t >= I.nTF) return;
    const R *fmac = (const R *)F.if_mac;
    const R *hm = (const R *)I.hist_m;
    signed char kind[3][2];
    int ref[3][2];
#pragma unroll
    for (int b = 0; b < D; b++)
#pragma unroll
        for (int s = 0; s < 2; s++) {
            const int k = t * 2 * D + 2 * b + s;
            kind[b][s] = I.tf_rkind[k];
            ref[b][s] = I.tf_ridx[k];
        }
    R rho[3][2], u[3][2][3];
#pragma unroll
    for (int b = 0; b < D; b++)
#pragma unroll
        for (int s = 0; s < 2; s++) {
            const int kd = kind[b][s], rf = ref[b][s];
            R r = R(0), m[3] = {R(0), R(0), R(0)};
            if (kd == RK_FINE) {
                // post-stream moments of the fine neighbour
                const int x = rf % F.g.n[0], yz = rf / F.g.n[0];
                const int y = yz % F.g.n[1], z = yz / F.g.n[1];
                static_for<Q>([&](auto ic) {
                    constexpr int i = decltype(ic)::value;
                    const int src = nb_index(F.g, x, y, z, -L::c(i, 0), -L::c(i, 1), -L::c(i, 2));
                    const R v = src >= 0 ? St<S>::ld(ff, (long long)i * F.g.pitch + src, F.g.shift[i]) : R(0);
                    r += v;
                    static_for<D>([&](auto ac) {
                        constexpr int a = decltype(ac)::value;
                        if constexpr (L::c(i, a) > 0) m[a] += v;
                        else if constexpr (L::c(i, a) < 0) m[a] -= v;
                    });
                });
#pragma unroll
                for (int a = 0; a < D; a++) m[a] /= r;
            } else if (kd == RK_TF) {
                r = fmac[rf];
#pragma unroll
                for (int a = 0; a < D; a++) m[a] = fmac[(long long)(1 + a) * F.nif + rf];
            } else {
#pragma unroll
                for (int j = 0; j < 3; j++) {
                    if (!((tw.nz >> j) & 1)) continue;
                    const R *h = hm + (long long)tw.slot[j] * 4 * I.nRing;
                    const R wj = tw_w<R>(tw, j);
                    r += wj * h[rf];
#pragma unroll
                    for (int a = 0; a < D; a++) m[a] += wj * h[(long long)(1 + a) * I.nRing + rf];
                }
            }
            rho[b][s] = r;
#pragma unroll
            for (int a = 0; a < 3; a++) u[b][s][a] = a < D ? m[a] : R(0);
        }
    R Sg[6], Cg[6];
    fd_gradients<D, R>(rho, u, R(0.5), Sg, Cg);  // coarse units: neighbours one coarse cell away
    R *fS = (R *)F.if_S, *fC = (R *)F.if_C;
#pragma unroll
    for (int k = 0; k < 6; k++) {
        fS[(long long)k * F.nif + t] = R(0.5) * Sg[k];
        fC[(long long)k * F.nif + t] = R(0.5) * Cg[k];
        if (sync) {
            ((R *)Cl.if_S)[(long long)k * Cl.nif + I.tfc_base + t] = Sg[k];
            ((R *)Cl.if_C)[(long long)k * Cl.nif + I.tfc_base + t] = Cg[k];
        }
    }
}

// ------------------------------------------------------------------ hanging nodes
// 4-point 1-D Lagrange along the interface (tensor order over odd axes, one-sided
// next to corners) of missing populations; macros are the moments.  One hanging node
// per thread.  S and C of hanging nodes are interpolated with the same stencil by the
// 2-D tile kernel where they are used (collide_store) and for D3Q19 by k_ie_sc after
// this launch.
template <int Q, typename S>
__device__ __forceinline__ void ie_node(int bid, IfaceDev I, LevelDev F, const S *__restrict__ ff)
{
    using L = Lat<Q>;
    using R = typename St<S>::R;
    constexpr int D = L::D;
    const int e = bid * blockDim.x + threadIdx.x;
    if (e >= I.nIE) return;
    const int nif = F.nif;
    const int row = I.nTF + e;  // table index of this hanging node
    R *fpop = (R *)F.if_pop;
    const R *iw = (const R *)I.ie_w;
    const unsigned kfm = I.ie_kf[e];
    const int nst = I.ie_nst[e];
    const int x = I.ie_f[3 * e], y = I.ie_f[3 * e + 1], z = I.ie_f[3 * e + 2];
    // the stencil slots in registers once: the gathers of every missing population are
    // then independent loads (the table stores between populations would otherwise
    // force the slots to be read again after each)
    constexpr int NS = kIeSlots<D>;
    int st[NS];
    R w[NS];
#pragma unroll
    for (int k = 0; k < NS; k++) {
        st[k] = I.ie_st[e * 16 + k];
        w[k] = iw[e * 16 + k];
    }
    R rho = R(0), m[3] = {R(0), R(0), R(0)};
    static_for<Q>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        R v = R(0);
        if ((kfm >> i) & 1u) {
            const int s = nb_index(F.g, x, y, z, -L::c(i, 0), -L::c(i, 1), -L::c(i, 2));
            if (s >= 0) v = St<S>::ld(ff, (long long)i * F.g.pitch + s, F.g.shift[i]);
        } else {
#pragma unroll
            for (int k = 0; k < NS; k++)
                if (k < nst) v += w[k] * fpop[(long long)i * nif + st[k]];
        }
        fpop[(long long)i * nif + row] = v;
        rho += v;
        static_for<D>([&](auto ac) {
            constexpr int a = decltype(ac)::value;
            if constexpr (L::c(i, a) > 0) m[a] += v;
            else if constexpr (L::c(i, a) < 0) m[a] -= v;
        });
    });
    R *fmac = (R *)F.if_mac;
    fmac[row] = rho;
#pragma unroll
    for (int a = 0; a < 3; a++) fmac[(long long)(1 + a) * nif + row] = a < D ? m[a] / rho : R(0);
}

// ------------------------------------------------------------------ launch chaining
// Programmatic dependent launch: the schedule's kernels first wait until the previous
// kernel of their stream has completed and flushed its memory (a no-op for a launch
// without the attribute), then allow the next kernel to start launching, so that its
// launch and block scheduling overlap this kernel's run.
__device__ __forceinline__ void pdl_enter()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// ------------------------------------------------------------------ fused launches
// blocks [0, nb_a) run the first body, the rest the second: the two halves work on
// independent data (a different interface, or TF nodes vs hanging nodes of the same
// interface whose inputs were all written by earlier launches).  NODE selects one node
// per thread (large interfaces) or one W-lane segment per node (small ones).
template <int Q, typename S, bool NODE>
__global__ void __launch_bounds__(128) k_recon_hist(const __grid_constant__ IfaceDev Ir, const __grid_constant__ LevelDev F,
                                                      const __grid_constant__ LevelDev Cl, const S *__restrict__ ff,
                                                      const __grid_constant__ TimeW tw, int sync, int *status, int *max_iters,
                                                      int nb_recon, const __grid_constant__ IfaceDev Ih,
                                                      const __grid_constant__ LevelGeo gh, const S *__restrict__ fh, int slot)
{
    pdl_enter();
    if ((int)blockIdx.x < nb_recon) {
        if constexpr (NODE) recon_node<Q, S>(blockIdx.x, Ir, F, Cl, ff, tw, sync, status, max_iters);
        else recon_seg<Q, S>(blockIdx.x, Ir, F, Cl, ff, tw, sync, status, max_iters);
    } else {
        if constexpr (NODE) hist_node<Q, S>(blockIdx.x - nb_recon, Ih, gh, fh, slot, 0);
        else hist_seg<Q, S>(blockIdx.x - nb_recon, Ih, gh, fh, slot, 0);
    }
}

template <int Q, typename S>
__global__ void __launch_bounds__(128) k_hist(const __grid_constant__ IfaceDev I, const __grid_constant__ LevelGeo gc,
                                             const S *__restrict__ fc, int slot, int seed)
{
    hist_node<Q, S>(blockIdx.x, I, gc, fc, slot, seed);
}

template <int Q, typename S, bool NODE>
__global__ void __launch_bounds__(128) k_grad_ie(const __grid_constant__ IfaceDev I, const __grid_constant__ LevelDev F,
                                                   const __grid_constant__ LevelDev Cl, const S *__restrict__ ff,
                                                   const __grid_constant__ TimeW tw, int sync, int nb_grad)
{
    pdl_enter();
    if ((int)blockIdx.x < nb_grad) {
        if constexpr (NODE) grad_node<Q, S>(blockIdx.x, I, F, Cl, ff, tw, sync);
        else grad_seg<Q, S>(blockIdx.x, I, F, Cl, ff, tw, sync);
    } else {
        if constexpr (NODE) ie_node<Q, S>(blockIdx.x - nb_grad, I, F, ff);
        else ie_seg<Q, S>(blockIdx.x - nb_grad, I, F, ff);
    }
}

// S and C of the hanging nodes of a level (D3Q19): the same 4-point stencils over the
// level's TF rows as their missing populations (tensor order over the node's odd axes,
// up to 16 points), written to the hanging nodes' own table rows, so that the bulk
// collision reads them like a TF node's.  One hanging node per thread; launched after
// the gradient launch that writes the TF rows.  The sum runs in stencil order, as the
// 2-D tile kernel's in-place interpolation does.
template <typename R>
__global__ void __launch_bounds__(128) k_ie_sc(const __grid_constant__ LevelDev F)
{
    pdl_enter();
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= F.n_ie) return;
    R *tS = (R *)F.if_S, *tC = (R *)F.if_C;
    const int nst = F.ie_nst[e];
    int st[16];
    R w[16];
#pragma unroll
    for (int j = 0; j < 16; j++) {
        st[j] = F.ie_st[e * 16 + j];
        w[j] = ((const R *)F.ie_w)[e * 16 + j];
    }
    R Sv[6], Cv[6];
#pragma unroll
    for (int q = 0; q < 6; q++) Sv[q] = Cv[q] = R(0);
#pragma unroll
    for (int j = 0; j < 16; j++) {
        if (j < nst) {
#pragma unroll
            for (int q = 0; q < 6; q++) {
                Sv[q] += w[j] * tS[(long long)q * F.nif + st[j]];
                Cv[q] += w[j] * tC[(long long)q * F.nif + st[j]];
            }
        }
    }
    const long long row = F.ie_base + e;
#pragma unroll
    for (int q = 0; q < 6; q++) {
        tS[(long long)q * F.nif + row] = Sv[q];
        tC[(long long)q * F.nif + row] = Cv[q];
    }
}

// ------------------------------------------------------------------ bulk collide-and-stream
// Tile class from the box geometry alone (no memory access): FAST when the tile
// grown by two nodes stays inside the band of bulk nodes (off the level's own outline,
// off the closed child box, no periodic wrap), SKIP when every node of the tile lies
// strictly inside the child box (the hole), GENERAL otherwise.  The host checks at
// creation that this rule reproduces the node-by-node classification of every tile.
template <int D>
__device__ __forceinline__ unsigned char tile_class(const LevelDev &Lv, const int *t0, const int *T)
{
    bool fast = true;
#pragma unroll
    for (int a = 0; a < D; a++)
        if (t0[a] - 2 < Lv.fast_lo[a] || t0[a] + T[a] + 1 > Lv.fast_hi[a]) fast = false;
    if (Lv.has_child) {
        bool disjoint = false, in_hole = true;
#pragma unroll
        for (int a = 0; a < D; a++) {
            if (Lv.child_per[a]) continue;
            if (t0[a] + T[a] + 1 < Lv.child_lo[a] || t0[a] - 2 > Lv.child_hi[a]) disjoint = true;
            const int last = min(t0[a] + T[a] - 1, Lv.g.n[a] - 1);
            if (!(t0[a] > Lv.child_lo[a] && last < Lv.child_hi[a])) in_hole = false;
        }
        if (in_hole) return TILE_SKIP;
        if (!disjoint) fast = false;
    }
    return fast ? TILE_FAST : TILE_GENERAL;
}

// post-stream moments of populations held in registers
template <int Q, typename R>
__device__ __forceinline__ void reg_moments(const R (&f)[Q], R &rho, R *u)
{
    using L = Lat<Q>;
    constexpr int D = L::D;
    R r = R(0), m[3] = {R(0), R(0), R(0)};
    static_for<Q>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        r += f[i];
        static_for<D>([&](auto ac) {
            constexpr int a = decltype(ac)::value;
            if constexpr (L::c(i, a) > 0) m[a] += f[i];
            else if constexpr (L::c(i, a) < 0) m[a] -= f[i];
        });
    });
    rho = r;
    const R inv = recip(r);
#pragma unroll
    for (int a = 0; a < D; a++) u[a] = m[a] * inv;
}

// Collision of one node from the shared-memory macros (bulk) or the interface table,
// then the store.
template <int Q, typename S, int HX, int HY, int HPLANE>
__device__ __forceinline__ void collide_store(const LevelDev &Lv, typename St<S>::R (&f)[Q], typename St<S>::R rho,
                                              const typename St<S>::R *u, int tag, int hself,
                                              const typename St<S>::R *s_rho, const typename St<S>::R *s_u,
                                              typename St<S>::R tau, typename St<S>::R om, typename St<S>::R sigma,
                                              typename St<S>::R spsi, S *__restrict__ fdst, int idx)
{
    using L = Lat<Q>;
    using R = typename St<S>::R;
    constexpr int D = L::D;
    R Sv[6], Cv[6];
    if (tag == TAG_BULK) {
        R nr[3][2], nu[3][2][3];
#pragma unroll
        for (int b = 0; b < D; b++)
#pragma unroll
            for (int s2 = 0; s2 < 2; s2++) {
                const int o = (s2 == 0 ? 1 : -1);
                const int hh = hself + (b == 0 ? o : (b == 1 ? o * HX : o * HX * HY));
                nr[b][s2] = s_rho[hh];
#pragma unroll
                for (int a = 0; a < D; a++) nu[b][s2][a] = s_u[a * HPLANE + hh];
                if (D == 2) nu[b][s2][2] = R(0);
            }
        fd_gradients<D, R>(nr, nu, R(0.5), Sv, Cv);
    } else if (tag >= Lv.ie_base && tag < Lv.ie_base + Lv.n_ie) {
        // hanging node: S and C by the same stencil as its missing populations (D2Q9:
        // 4 or 2 points along the interface).  The stencil rows are [n_ie][16], so the
        // four slots are read at once with the count, then the table rows of the used
        // slots at once: two dependent round trips instead of two per point
        static_assert(L::D == 2, "2-D stencils have at most 4 points");
        const R *tS = (const R *)Lv.if_S, *tC = (const R *)Lv.if_C;
        const int e = tag - Lv.ie_base, nst = Lv.ie_nst[e];
        int tf[4];
        R wj[4];
#pragma unroll
        for (int j = 0; j < 4; j++) {
            tf[j] = Lv.ie_st[e * 16 + j];
            wj[j] = ((const R *)Lv.ie_w)[e * 16 + j];
        }
#pragma unroll
        for (int k = 0; k < 6; k++) {
            Sv[k] = R(0);
            Cv[k] = R(0);
        }
#pragma unroll
        for (int j = 0; j < 4; j++) {
            if (j >= nst) break;
#pragma unroll
            for (int k = 0; k < 6; k++) {
                Sv[k] += wj[j] * tS[(long long)k * Lv.nif + tf[j]];
                Cv[k] += wj[j] * tC[(long long)k * Lv.nif + tf[j]];
            }
        }
    } else {
        const R *tS = (const R *)Lv.if_S, *tC = (const R *)Lv.if_C;
#pragma unroll
        for (int k = 0; k < 6; k++) {
            Sv[k] = tS[(long long)k * Lv.nif + tag];
            Cv[k] = tC[(long long)k * Lv.nif + tag];
        }
    }
    hrr_collide<Q, R>(f, rho, u, Sv, Cv, tau, om, sigma, spsi);
    static_for<Q>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        St<S>::st(fdst + (long long)i * Lv.g.pitch, idx, f[i], Lv.g.shift[i]);
    });
}

// 2-D: one CTA per tile of TX x (TYT*NR) nodes, TX x TYT threads, NR nodes per thread
// (rows ty, ty+TYT, ...).  Every node of the tile and of its one-node halo pulls its
// post-stream populations (or reads them from the interface table) and leaves rho, u
// in shared memory; every tile node then takes centred differences from its
// neighbours (or the supplied S, C of interface nodes) and collides.  The
// 2(TX+TY)+4 halo nodes are shared out one per thread; all loads of a thread (its
// nodes and its halo node) go out before any is used.
// NBUF = 2 keeps two sets of the shared macro arrays (buf = 0, 1): a CTA that runs
// tiles back to back alternates them after every tile that returned true (a tile
// that passed its barrier) and needs no barrier between tiles.  Returns false for a
// skipped tile.
template <int Q, typename S, int TX, int TYT, int NR, int NBUF = 1>
__device__ __forceinline__ bool bulk2d_tile(const LevelDev &Lv, const S *__restrict__ fsrc, S *__restrict__ fdst,
                                            typename St<S>::R tau, typename St<S>::R om, typename St<S>::R sigma,
                                            typename St<S>::R spsi, int bx, int by, int buf = 0)
{
    using L = Lat<Q>;
    using R = typename St<S>::R;
    constexpr int D = 2;
    static_assert(L::D == 2, "2-D kernel");
    constexpr int TY = TYT * NR;
    constexpr int HX = TX + 2, HY = TY + 2;
    constexpr int H = HX * HY;
    constexpr int NT = TX * TYT;
    constexpr int NB = 2 * HX + 2 * TY;  // halo positions
    static_assert(NB <= NT, "one halo node per thread at most");
    __shared__ R s_rho_all[NBUF][H];
    __shared__ R s_u_all[NBUF][D * H];
    R *s_rho = s_rho_all[NBUF > 1 ? buf : 0];
    R *s_u = s_u_all[NBUF > 1 ? buf : 0];
    const LevelGeo &g = Lv.g;
    const int X0 = bx * TX, Y0 = by * TY;
    const int t0[3] = {X0, Y0, 0}, T[3] = {TX, TY, 1};
    const unsigned char flag =
        Lv.tile_flags ? Lv.tile_flags[bx + ((Lv.g.n[0] + TX - 1) / TX) * by] : tile_class<D>(Lv, t0, T);
    if (flag == TILE_SKIP) return false;
    const int tid = threadIdx.x;
    const int tx = tid % TX, tr = tid / TX;
    const int x = X0 + tx;

    // halo position owned by this thread
    int hb = -1, hx = 0, hy = 0;
    if (tid < NB) {
        if (tid < HX) {
            hx = tid;
            hy = 0;
        } else if (tid < 2 * HX) {
            hx = tid - HX;
            hy = HY - 1;
        } else {
            const int b = tid - 2 * HX;
            hy = 1 + (b >> 1);
            hx = (b & 1) ? HX - 1 : 0;
        }
        hb = hx + HX * hy;
    }

    R f[NR][Q], fh[Q];
    int tag[NR];
    int htag = TAG_HOLE;
    bool inside[NR];
    int idx[NR];
#pragma unroll
    for (int r = 0; r < NR; r++) {
        const int y = Y0 + tr + r * TYT;
        inside[r] = x < g.n[0] && y < g.n[1];
        idx[r] = x + g.px * y;
    }
    int otag[NR];
    if (flag == TILE_FAST) {
#pragma unroll
        for (int r = 0; r < NR; r++) otag[r] = TAG_BULK;
        htag = hb >= 0 ? TAG_BULK : TAG_HOLE;
        const int hidx = (X0 + hx - 1) + g.px * (Y0 + hy - 1);
#pragma unroll
        for (int i = 0; i < Q; i++) {
            const S *pi = fsrc + (long long)i * g.pitch;  // population plane
            const int off = L::c(i, 0) + g.px * L::c(i, 1);
#pragma unroll
            for (int r = 0; r < NR; r++) f[r][i] = St<S>::ld(pi, idx[r] - off, g.shift[i]);
        }
        if (hb >= 0) {
#pragma unroll
            for (int i = 0; i < Q; i++) {
                const int off = L::c(i, 0) + g.px * L::c(i, 1);
                fh[i] = St<S>::ld(fsrc + (long long)i * g.pitch, hidx - off, g.shift[i]);
            }
        }
    } else {
        // own positions (wrapped when a ragged tile sits past a periodic seam) and the
        // halo position: their tags, and with them every bulk pull of a position inside
        // the box (a bulk node's sources are nodes, reached with a one-step wrap on
        // periodic axes; for any other position inside the box the same one-step wrap
        // keeps the address inside the box, and its value is replaced below), so that a
        // bulk node of a general tile waits for one round trip, not two
        int ox[NR], oy[NR];
        bool okp[NR];
#pragma unroll
        for (int r = 0; r < NR; r++) {
            ox[r] = x;
            oy[r] = Y0 + tr + r * TYT;
            okp[r] = wrap_coord(ox[r], g.n[0], g.per[0]) && wrap_coord(oy[r], g.n[1], g.per[1]);
            otag[r] = okp[r] ? Lv.tag[ox[r] + g.px * oy[r]] : TAG_HOLE;
        }
        int qx = X0 + hx - 1, qy = Y0 + hy - 1;
        const bool hvalid = hb >= 0 && wrap_coord(qx, g.n[0], g.per[0]) && wrap_coord(qy, g.n[1], g.per[1]);
        htag = hvalid ? Lv.tag[qx + g.px * qy] : TAG_HOLE;
#pragma unroll
        for (int i = 0; i < Q; i++) {
            const S *pi = fsrc + (long long)i * g.pitch;
#pragma unroll
            for (int r = 0; r < NR; r++) {
                int sx = ox[r] - L::c(i, 0), sy = oy[r] - L::c(i, 1);
                sx += (sx < 0) ? g.n[0] : ((sx >= g.n[0]) ? -g.n[0] : 0);
                sy += (sy < 0) ? g.n[1] : ((sy >= g.n[1]) ? -g.n[1] : 0);
                f[r][i] = okp[r] ? St<S>::ld(pi, sx + g.px * sy, g.shift[i]) : R(0);
            }
            int hsx = qx - L::c(i, 0), hsy = qy - L::c(i, 1);
            hsx += (hsx < 0) ? g.n[0] : ((hsx >= g.n[0]) ? -g.n[0] : 0);
            hsy += (hsy < 0) ? g.n[1] : ((hsy >= g.n[1]) ? -g.n[1] : 0);
            fh[i] = hvalid ? St<S>::ld(pi, hsx + g.px * hsy, g.shift[i]) : R(0);
        }
        // positions that are not bulk nodes: table rows (interface) or nothing (hole)
        const R *pop = (const R *)Lv.if_pop;
#pragma unroll
        for (int r = 0; r < NR; r++)
            if (otag[r] != TAG_BULK) {
#pragma unroll
                for (int i = 0; i < Q; i++) f[r][i] = otag[r] >= 0 ? pop[(long long)i * Lv.nif + otag[r]] : R(0);
            }
        if (htag != TAG_BULK) {
#pragma unroll
            for (int i = 0; i < Q; i++) fh[i] = htag >= 0 ? pop[(long long)i * Lv.nif + htag] : R(0);
        }
    }
    // macros of every own position (a position past a periodic seam stands for the
    // wrapped node) and of the halo position
    R rho[NR], u[NR][3];
    const R *mac = (const R *)Lv.if_mac;
#pragma unroll
    for (int r = 0; r < NR; r++) {
        rho[r] = R(1);
        u[r][0] = u[r][1] = u[r][2] = R(0);
        if (otag[r] == TAG_BULK) {
            reg_moments<Q, R>(f[r], rho[r], u[r]);
        } else if (otag[r] >= 0) {
            rho[r] = mac[otag[r]];
#pragma unroll
            for (int a = 0; a < D; a++) u[r][a] = mac[(long long)(1 + a) * Lv.nif + otag[r]];
        }
        tag[r] = inside[r] ? otag[r] : TAG_HOLE;
        const int hs = (tx + 1) + HX * (tr + r * TYT + 1);
        s_rho[hs] = rho[r];
#pragma unroll
        for (int a = 0; a < D; a++) s_u[a * H + hs] = u[r][a];
    }
    if (hb >= 0) {
        R hr = R(1), hu[3] = {R(0), R(0), R(0)};
        if (htag == TAG_BULK) {
            reg_moments<Q, R>(fh, hr, hu);
        } else if (htag >= 0) {
            hr = mac[htag];
#pragma unroll
            for (int a = 0; a < D; a++) hu[a] = mac[(long long)(1 + a) * Lv.nif + htag];
        }
        s_rho[hb] = hr;
#pragma unroll
        for (int a = 0; a < D; a++) s_u[a * H + hb] = hu[a];
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < NR; r++) {
        if (tag[r] == TAG_HOLE) continue;
        const int hs = (tx + 1) + HX * (tr + r * TYT + 1);
        collide_store<Q, S, HX, HY, H>(Lv, f[r], rho[r], u[r], tag[r], hs, s_rho, s_u, tau, om, sigma, spsi, fdst,
                                       idx[r]);
    }
    return true;
}

template <int Q, typename S, int TX, int TYT, int NR>
__global__ void __launch_bounds__(TX *TYT, sizeof(S) == 8 ? 1 : (TX * TYT >= 256 ? 1024 / (TX * TYT) : 4)) k_bulk2d(const __grid_constant__ LevelDev Lv, const S *__restrict__ fsrc, S *__restrict__ fdst,
                                                     typename St<S>::R tau, typename St<S>::R om,
                                                     typename St<S>::R sigma, typename St<S>::R spsi)
{
    pdl_enter();
    bulk2d_tile<Q, S, TX, TYT, NR>(Lv, fsrc, fdst, tau, om, sigma, spsi, blockIdx.x, blockIdx.y);
}

// Geometric class of one plane p of a z-marching tile: LOAD_FAST when the tile grown by
// two nodes in x and y, over planes p-1..p+1, lies in the band of bulk nodes (its own
// nodes and their halo are bulk, all their sources are nodes without periodic wrap);
// LOAD_HOLE when the tile grown by one node in x and y lies strictly inside the child
// box at plane p (nothing to load); LOAD_GENERAL otherwise.
enum : int { LOAD_FAST = 0, LOAD_HOLE = 1, LOAD_GENERAL = 2 };

__device__ __forceinline__ int plane_class(const LevelDev &Lv, int X0, int Y0, int TX, int TY, int p)
{
    const int lo[3] = {X0 - 2, Y0 - 2, p - 1}, hi[3] = {X0 + TX + 1, Y0 + TY + 1, p + 1};
    bool fast = true;
#pragma unroll
    for (int a = 0; a < 3; a++)
        if (lo[a] < Lv.fast_lo[a] || hi[a] > Lv.fast_hi[a]) fast = false;
    if (Lv.has_child) {
        bool disjoint = false, in_hole = true;
        const int hlo[3] = {X0 - 1, Y0 - 1, p}, hhi[3] = {min(X0 + TX, Lv.g.n[0] - 1), min(Y0 + TY, Lv.g.n[1] - 1), p};
#pragma unroll
        for (int a = 0; a < 3; a++) {
            if (Lv.child_per[a]) continue;
            if (hi[a] < Lv.child_lo[a] || lo[a] > Lv.child_hi[a]) disjoint = true;
            if (!(hlo[a] > Lv.child_lo[a] && hhi[a] < Lv.child_hi[a])) in_hole = false;
        }
        if (in_hole) return LOAD_HOLE;
        if (!disjoint) fast = false;
    }
    return fast ? LOAD_FAST : LOAD_GENERAL;
}

// plane_class with its x-y half evaluated once for a column: per plane only the z
// intervals remain (the same classes, fewer instructions per plane)
struct PlaneRule {
    bool fxy, child, disj_xy, hole_xy, zper;
    int zflo, zfhi, zclo, zchi;
    __device__ __forceinline__ PlaneRule(const LevelDev &Lv, int X0, int Y0, int TX, int TY)
    {
        const int lo[2] = {X0 - 2, Y0 - 2}, hi[2] = {X0 + TX + 1, Y0 + TY + 1};
        fxy = true;
#pragma unroll
        for (int a = 0; a < 2; a++)
            if (lo[a] < Lv.fast_lo[a] || hi[a] > Lv.fast_hi[a]) fxy = false;
        zflo = Lv.fast_lo[2];
        zfhi = Lv.fast_hi[2];
        child = Lv.has_child != 0;
        disj_xy = false;
        hole_xy = true;
        if (child) {
            const int hlo[2] = {X0 - 1, Y0 - 1}, hhi[2] = {min(X0 + TX, Lv.g.n[0] - 1), min(Y0 + TY, Lv.g.n[1] - 1)};
#pragma unroll
            for (int a = 0; a < 2; a++) {
                if (Lv.child_per[a]) continue;
                if (hi[a] < Lv.child_lo[a] || lo[a] > Lv.child_hi[a]) disj_xy = true;
                if (!(hlo[a] > Lv.child_lo[a] && hhi[a] < Lv.child_hi[a])) hole_xy = false;
            }
        }
        zper = Lv.child_per[2] != 0;
        zclo = Lv.child_lo[2];
        zchi = Lv.child_hi[2];
    }
    __device__ __forceinline__ int operator()(int p) const
    {
        bool fast = fxy && p - 1 >= zflo && p + 1 <= zfhi;
        if (child) {
            const bool disj = disj_xy || (!zper && (p + 1 < zclo || p - 1 > zchi));
            if (hole_xy && (zper || (p > zclo && p < zchi))) return LOAD_HOLE;
            if (!disj) fast = false;
        }
        return fast ? LOAD_FAST : LOAD_GENERAL;
    }
};

__device__ __forceinline__ unsigned long long globaltimer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// ------------------------------------------------------------------ bulk tensor copies
// The tensor map of a 3-D population buffer is 4-D: x (n[0], contiguous), y (stride
// px), z (stride px n[1]) and the population index (stride pitch).  One copy moves the
// box of one population over TX+2XA x TY+4 nodes of one plane into shared memory and
// signals an mbarrier with its byte count.
namespace tma {
__device__ __forceinline__ unsigned saddr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(saddr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// the same test, suspending the thread until the phase completes or about hint_ns
// nanoseconds have passed (a waiting warp sleeps instead of spinning)
__device__ __forceinline__ bool mbar_try_wait_hint(unsigned long long *bar, unsigned parity, unsigned hint_ns)
{
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\tselp.u32 %0, 1, 0, "
        "p;\n\t}"
        : "=r"(ok)
        : "r"(saddr(bar)), "r"(parity), "r"(hint_ns)
        : "memory");
    return ok != 0;
}
// wait for the phase with the given parity, at most limit_ns; false on time-out
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity, unsigned long long limit_ns)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = globaltimer_ns();
    while (!mbar_try_wait_hint(bar, parity, 100000u))
        if (globaltimer_ns() - t0 > limit_ns) return false;
    return true;
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// copy global -> shared without the register file (4, 8 or 16 bytes, both addresses
// aligned to the size; zero-fill when !ok)
template <int B>
__device__ __forceinline__ void cp_async(void *dst, const void *src, bool ok)
{
    static_assert(B == 4 || B == 8 || B == 16, "cp.async size");
    if constexpr (B == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(saddr(dst)), "l"(src), "r"(ok ? 16 : 0)
                     : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;" ::"r"(saddr(dst)), "l"(src), "n"(B),
                     "r"(ok ? B : 0)
                     : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
__device__ __forceinline__ void load4d(void *dst, const CUtensorMap *map, unsigned long long *bar, int c0, int c1,
                                       int c2, int c3)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5, %6}], "
        "[%2];" ::"r"(saddr(dst)),
        "l"(map), "r"(saddr(bar)), "r"(c0), "r"(c1), "r"(c2), "r"(c3)
        : "memory");
}
}  // namespace tma

// ------------------------------------------------------------------ batched persistent launch
// Many independent hierarchies with the same number of levels advance together: the
// sub-cycle schedule of one coarse step is a list of phases (history + Newton,
// gradients + hanging nodes, bulk) and every phase is one grid-stride pass over the
// work items of all hierarchies.  One cooperative launch runs all phases of n coarse
// steps with a grid barrier between dependent phases.
enum : int { PH_RH = 0, PH_GI = 1, PH_BULK = 2 };

struct BatchPhase {
    int kind, level, sub;  // level step index k_l = k * 2^level + sub for coarse step k
    int join_next;         // the next phase is independent of this one: no barrier between
};

struct BatchDev {
    int n, L;
    const LevelDev *lev;    // [n][L]
    const IfaceDev *ifc;    // [n][L]; ifc[h*L + l] couples levels l-1 and l
    const int *pre_bulk;    // [L][n+1] prefix sums of bulk tiles
    const int *pre_rh;      // [L][n+1] prefix sums of (Newton + history) blocks
    const int *nb_recon;    // [L][n] Newton blocks of each hierarchy (the rest is history)
    const int *pre_gi;      // [L][n+1] prefix sums of (gradient + hanging) blocks
    const int *nb_grad;     // [L][n]
    const int *node_rh, *node_gi;  // [L][n] one node per thread (1) or one segment per node (0)
    int *status, *max_iters;
    unsigned int *bar_count, *bar_gen;
    unsigned long long barrier_ns;  // a barrier wait longer than this gives up
};

// Grid-wide barrier of a cooperative launch.  Thread 0 of each block arrives on a
// counter; the last arrival resets it and bumps the generation; the others wait for
// the generation to change, at most limit_ns, after which they set ST_TIMEOUT and the
// barrier returns false (the caller stops).
__device__ __forceinline__ bool grid_barrier(unsigned int *count, unsigned int *gen, unsigned int nblocks,
                                             int *status, unsigned long long limit_ns)
{
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        volatile unsigned int *vgen = gen;
        const unsigned int g0 = *vgen;
        __threadfence();
        if (atomicAdd(count, 1u) == nblocks - 1) {
            *((volatile unsigned int *)count) = 0u;
            __threadfence();
            atomicAdd(gen, 1u);
        } else {
            const unsigned long long t0 = globaltimer_ns();
            while (*vgen == g0) {
                if (globaltimer_ns() - t0 > limit_ns) {
                    atomicOr(status, ST_TIMEOUT);
                    ok = 0;
                    break;
                }
                __nanosleep(100);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

// hierarchy owning work item t: the last h with pre[h] <= t
__device__ __forceinline__ int owner(const int *pre, int n, int t)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (pre[mid] <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ TimeW batch_weights(int phase, long long kp) { return time_weights(phase, kp); }

// Phase bodies of the batched kernel as separate (not inlined) functions: each gets
// its own register allocation instead of the union of all phases.
template <int Q, typename S, int TX, int TYT, int NR>
__device__ __forceinline__ bool batch_bulk_tile(const LevelDev &Lv, long long kl, int local, int buf)
{
    using R = typename St<S>::R;
    const bool dbl = sizeof(R) == 8;
    return bulk2d_tile<Q, S, TX, TYT, NR, 2>(Lv, (const S *)Lv.f[kl & 1], (S *)Lv.f[(kl + 1) & 1],
                                      dbl ? (R)Lv.tau : (R)Lv.tauf, dbl ? (R)Lv.om : (R)Lv.omf,
                                      dbl ? (R)Lv.sigma : (R)Lv.sigmaf, dbl ? (R)Lv.spsi : (R)Lv.spsif,
                                      local % Lv.tiles[0], local / Lv.tiles[0], buf);
}
template <int Q, typename S>
__device__ __noinline__ void batch_recon_hist(const BatchDev &B, int h, int l, long long kl, int local, TimeW tw)
{
    const int nbr = B.nb_recon[(size_t)l * B.n + h];
    const bool node = B.node_rh[(size_t)l * B.n + h] != 0;
    const LevelDev &F = B.lev[h * B.L + l];
    const S *fA = (const S *)F.f[kl & 1];
    if (local < nbr) {
        if (node)
            recon_node<Q, S>(local, B.ifc[h * B.L + l], F, B.lev[h * B.L + l - 1], fA, tw, (int)(kl & 1), B.status,
                             B.max_iters);
        else
            recon_seg<Q, S>(local, B.ifc[h * B.L + l], F, B.lev[h * B.L + l - 1], fA, tw, (int)(kl & 1), B.status,
                            B.max_iters);
    } else {
        if (node) hist_node<Q, S>(local - nbr, B.ifc[h * B.L + l + 1], F.g, fA, (int)((kl + 1) % 3), 0);
        else hist_seg<Q, S>(local - nbr, B.ifc[h * B.L + l + 1], F.g, fA, (int)((kl + 1) % 3), 0);
    }
}
template <int Q, typename S>
__device__ __noinline__ void batch_grad_ie(const BatchDev &B, int h, int l, long long kl, int local, TimeW tw)
{
    const int nbg = B.nb_grad[(size_t)l * B.n + h];
    const bool node = B.node_gi[(size_t)l * B.n + h] != 0;
    const LevelDev &F = B.lev[h * B.L + l];
    const S *fA = (const S *)F.f[kl & 1];
    if (local < nbg) {
        if (node) grad_node<Q, S>(local, B.ifc[h * B.L + l], F, B.lev[h * B.L + l - 1], fA, tw, (int)(kl & 1));
        else grad_seg<Q, S>(local, B.ifc[h * B.L + l], F, B.lev[h * B.L + l - 1], fA, tw, (int)(kl & 1));
    } else {
        if (node) ie_node<Q, S>(local - nbg, B.ifc[h * B.L + l], F, fA);
        else ie_seg<Q, S>(local - nbg, B.ifc[h * B.L + l], F, fA);
    }
}

// Registers: at 80 registers per thread three 256-thread CTAs share an SM (a tighter
// bound spills inside the tile body).
template <int Q, typename S, int TX, int TYT, int NR>
__global__ void __launch_bounds__(TX *TYT, sizeof(S) == 8 ? 1 : 3)
    k_batch(BatchDev B, const BatchPhase *__restrict__ phases, int nphases, long long k0, int nsteps)
{
    using R = typename St<S>::R;
    const unsigned int nb = gridDim.x;
    // the level view of the hierarchy whose tiles a CTA works on, copied to shared
    // memory when the CTA moves to another hierarchy or level
    __shared__ LevelDev s_lv;
    static_assert(sizeof(LevelDev) % 4 == 0, "word copy");
    for (int st = 0; st < nsteps; st++) {
        const long long k = k0 + st;
        for (int pi = 0; pi < nphases; pi++) {
            const BatchPhase ph = phases[pi];
            const int l = ph.level;
            const long long kl = (k << l) + ph.sub;
            if (ph.kind == PH_BULK) {
                const int *pre = B.pre_bulk + (size_t)l * (B.n + 1);
                int cur = -1, nbuf = 0;
                for (int t = blockIdx.x; t < pre[B.n]; t += nb) {
                    const int h = owner(pre, B.n, t);
                    if (h != cur) {
                        __syncthreads();  // the previous view is no longer read
                        const int *src = (const int *)&B.lev[h * B.L + l];
                        for (int w = threadIdx.x; w < (int)(sizeof(LevelDev) / 4); w += blockDim.x)
                            ((int *)&s_lv)[w] = src[w];
                        __syncthreads();
                        cur = h;
                    }
                    if (batch_bulk_tile<Q, S, TX, TYT, NR>(s_lv, kl, t - pre[h], nbuf))
                        nbuf ^= 1;  // alternate shared arrays: no barrier between tiles
                }
            } else if (ph.kind == PH_RH) {
                const int *pre = B.pre_rh + (size_t)l * (B.n + 1);
                const TimeW tw = l > 0 ? batch_weights((int)(kl & 1), kl >> 1) : TimeW{};
                for (int t = blockIdx.x; t < pre[B.n]; t += nb) {
                    const int h = owner(pre, B.n, t);
                    batch_recon_hist<Q, S>(B, h, l, kl, t - pre[h], tw);
                }
            } else {
                const int *pre = B.pre_gi + (size_t)l * (B.n + 1);
                const TimeW tw = batch_weights((int)(kl & 1), kl >> 1);
                for (int t = blockIdx.x; t < pre[B.n]; t += nb) {
                    const int h = owner(pre, B.n, t);
                    batch_grad_ie<Q, S>(B, h, l, kl, t - pre[h], tw);
                }
            }
            if (!ph.join_next && !grid_barrier(B.bar_count, B.bar_gen, nb, B.status, B.barrier_ns)) return;
        }
    }
}

// Phase-launch structure of a batch (the alternative to k_batch): every phase of the
// sub-cycle schedule is one ordinary launch with one CTA per work item of all members,
// so no CTA stays resident and no grid barrier is needed (kernel boundaries order
// dependent phases).  The bodies are the ones of k_batch: the results are bitwise the
// same.
template <int Q, typename S, int TX, int TYT, int NR>
__global__ void __launch_bounds__(TX *TYT, sizeof(S) == 8 ? 1 : (TX * TYT >= 256 ? 1024 / (TX * TYT) : 4))
    k_batch_bulk(BatchDev B, int l, long long kl)
{
    pdl_enter();
    using R = typename St<S>::R;
    __shared__ LevelDev s_lv;
    const int *pre = B.pre_bulk + (size_t)l * (B.n + 1);
    const int t = blockIdx.x;
    const int h = owner(pre, B.n, t);
    const int *src = (const int *)&B.lev[h * B.L + l];
    for (int w = threadIdx.x; w < (int)(sizeof(LevelDev) / 4); w += blockDim.x) ((int *)&s_lv)[w] = src[w];
    __syncthreads();
    const bool dbl = sizeof(R) == 8;
    const int local = t - pre[h];
    bulk2d_tile<Q, S, TX, TYT, NR, 1>(s_lv, (const S *)s_lv.f[kl & 1], (S *)s_lv.f[(kl + 1) & 1],
                                      dbl ? (R)s_lv.tau : (R)s_lv.tauf, dbl ? (R)s_lv.om : (R)s_lv.omf,
                                      dbl ? (R)s_lv.sigma : (R)s_lv.sigmaf, dbl ? (R)s_lv.spsi : (R)s_lv.spsif,
                                      local % s_lv.tiles[0], local / s_lv.tiles[0]);
}
template <int Q, typename S>
__global__ void __launch_bounds__(256) k_batch_rh(BatchDev B, int l, long long kl, TimeW tw)
{
    pdl_enter();
    const int *pre = B.pre_rh + (size_t)l * (B.n + 1);
    const int t = blockIdx.x;
    const int h = owner(pre, B.n, t);
    batch_recon_hist<Q, S>(B, h, l, kl, t - pre[h], tw);
}
template <int Q, typename S>
__global__ void __launch_bounds__(256) k_batch_gi(BatchDev B, int l, long long kl, TimeW tw)
{
    pdl_enter();
    const int *pre = B.pre_gi + (size_t)l * (B.n + 1);
    const int t = blockIdx.x;
    const int h = owner(pre, B.n, t);
    batch_grad_ie<Q, S>(B, h, l, kl, t - pre[h], tw);
}

// The barrier alone, for the bounded-wait check: with skip >= 0 that block returns
// without arriving, so every other block's wait runs out and sets ST_TIMEOUT.
__global__ void k_barrier_check(unsigned int *count, unsigned int *gen, int *status, unsigned long long limit_ns,
                                int skip)
{
    if ((int)blockIdx.x == skip) return;
    grid_barrier(count, gen, gridDim.x, status, limit_ns);
}


// ------------------------------------------------------------------ probes
// Density at probe points: (bi/tri)linear interpolation of rho over the 4 (8) nodes of
// the finest level whose cell holds the point; rho of a node is the zeroth moment of
// its current populations.  One thread per probe, one row of samples per call.
struct ProbeDev {
    int n;
    const int *level;     // [n]
    const int *node;      // [n][8] node indices in the level box
    const double *w;      // [n][8] weights
    double *samples;      // [capacity][n]
    int capacity;
};

template <int Q, typename S>
__global__ void k_probe(ProbeDev P, const LevelDev *__restrict__ levs, const long long *__restrict__ kstep, int row)
{
    using L = Lat<Q>;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= P.n || row >= P.capacity) return;
    const int l = P.level[j];
    const LevelDev &Lv = levs[l];
    const S *f = (const S *)Lv.f[kstep[l] & 1];
    double acc = 0.0;
    for (int c = 0; c < (L::D == 3 ? 8 : 4); c++) {
        const int idx = P.node[j * 8 + c];
        double r = 0.0;
        for (int i = 0; i < Q; i++) r += (double)St<S>::ld(f + (long long)i * Lv.g.pitch, idx, Lv.g.shift[i]);
        acc += P.w[j * 8 + c] * r;
    }
    P.samples[(long long)row * P.n + j] = acc;
}
// ------------------------------------------------------------------ utilities
template <int Q, typename S>
__global__ void k_init(LevelGeo g, const int *__restrict__ tag, const double *__restrict__ rho,
                       const double *__restrict__ u, S *__restrict__ f0, S *__restrict__ f1)
{
    using L = Lat<Q>;
    constexpr int D = L::D;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= g.N) return;
    const long long sl = dense_to_slot(g, idx);
    const bool hole = tag[sl] == TAG_HOLE;
    double uu[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < D; a++) uu[a] = u[(long long)a * g.N + idx];
#pragma unroll
    for (int i = 0; i < Q; i++) {
        const double v = hole ? L::w(i) : feq_one<Q>(i, rho[idx], uu);
        St<S>::st(f0, (long long)i * g.pitch + sl, (typename St<S>::R)v, g.shift[i]);
        St<S>::st(f1, (long long)i * g.pitch + sl, (typename St<S>::R)v, g.shift[i]);
    }
}

template <int Q, typename S>
__global__ void k_macros(LevelGeo g, const int *__restrict__ tag, const S *__restrict__ f, double *__restrict__ rho,
                         double *__restrict__ u, double *__restrict__ pops)
{
    using L = Lat<Q>;
    constexpr int D = L::D;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= g.N) return;
    const long long sl = dense_to_slot(g, idx);
    const bool hole = tag[sl] == TAG_HOLE;
    double r = 0.0, m[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int i = 0; i < Q; i++) {
        const double v = hole ? 0.0 : (double)St<S>::ld(f, (long long)i * g.pitch + sl, g.shift[i]);
        if (pops) pops[(long long)i * g.N + idx] = v;
        r += v;
        for (int a = 0; a < D; a++) m[a] += L::c(i, a) * v;
    }
    if (rho) rho[idx] = r;
    if (u)
        for (int a = 0; a < D; a++) u[(long long)a * g.N + idx] = hole ? 0.0 : m[a] / r;
}

// Sum of acc[0..3] over a block of 256 threads: warp shuffles within each warp, then
// the first warp over the 8 warp sums; the result is valid in thread 0 (fixed order,
// deterministic).
__device__ __forceinline__ void block_sum4_256(double (&acc)[4])
{
    __shared__ double sw[4][8];
#pragma unroll
    for (int k = 0; k < 4; k++)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_down_sync(0xffffffffu, acc[k], o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < 4; k++) sw[k][warp] = acc[k];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < 4; k++) {
            acc[k] = lane < 8 ? sw[k][lane] : 0.0;
#pragma unroll
            for (int o = 4; o > 0; o >>= 1) acc[k] += __shfl_down_sync(0xffffffffu, acc[k], o);
        }
    }
}

// Volume-weighted mass and momentum, per-block FP64 partials (deterministic order)
template <int Q, typename S>
__global__ void k_reduce_partial(LevelGeo g, const int *__restrict__ tag, const S *__restrict__ f,
                                 const double *__restrict__ wnode, double *__restrict__ partial, int *status)
{
    using L = Lat<Q>;
    constexpr int D = L::D;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    bool bad = false;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < g.N;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long sl = dense_to_slot(g, idx);
        if (tag[sl] == TAG_HOLE) continue;
        const double w = wnode[idx];
#pragma unroll
        for (int i = 0; i < Q; i++) {
            const double v = (double)St<S>::ld(f, (long long)i * g.pitch + sl, g.shift[i]);
            if (!isfinite(v)) bad = true;
            acc[0] += w * v;
            for (int a = 0; a < D; a++) acc[1 + a] += w * L::c(i, a) * v;
        }
    }
    if (bad) atomicOr(status, ST_NAN);
    block_sum4_256(acc);
    if (threadIdx.x == 0)
        for (int k = 0; k < 4; k++) partial[(long long)blockIdx.x * 4 + k] = acc[k];
}

__global__ void k_reduce_final(const double *__restrict__ partial, int nblocks, double *__restrict__ out)
{
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
        for (int k = 0; k < 4; k++) acc[k] += partial[(long long)b * 4 + k];
    block_sum4_256(acc);
    if (threadIdx.x == 0)
        for (int k = 0; k < 4; k++) out[k] = acc[k];
}

}  // namespace lbmg
