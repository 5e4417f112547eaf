// Kernels of the GB300 direct-coupling multi-level lattice Boltzmann library.
#pragma once

#include "lbm_device.cuh"

namespace lbmg {

// ------------------------------------------------------------------ interface views
struct IfaceDev {
    int nTF, nIE, nRing;
    // TF nodes: fine node index (level f), coarse node index (level c), population masks
    const long long *tf_fine;
    const long long *tf_coarse;
    const unsigned int *tf_kf;      // fine-known
    const unsigned int *tf_kc;      // coarse-known
    const unsigned int *tf_gc;      // gamma_i = c (Table 1)
    const signed char *tf_rkind;    // [nTF][2D] gradient stencil reference kind
    const long long *tf_ridx;       // [nTF][2D] reference index (fine node / TF / ring)
    // hanging nodes
    const long long *ie_fine;
    const unsigned int *ie_kf;
    const int *ie_nst;
    const int *ie_st;               // [nIE][16] TF indices
    const double *ie_w;             // [nIE][16]
    // ring of coarse stencil nodes
    const long long *ring_coarse;
    // history: coarse post-stream populations at TF [3][Q][nTF], ring macros [3][4][nRing]
    double *hist_f;
    double *hist_m;
    int tfc_base;                   // table index of the first TF node in the coarse level's table
    double R;                       // Eq. (fneqResc): R = tau_f / (2 tau_c)
};

struct TimeW {
    int slot[3];   // t - dt^c, t, t + dt^c
    double w[3];   // weights (Eq. TempInt, linear on the first coarse step, [0,0,1] on sync)
};

// ------------------------------------------------------------------ history push
// post-stream coarse populations at TF nodes (coarse-known ones) and post-stream
// macros at ring nodes, for the child level's Eq. (TempInt)
template <int Q, typename S>
__global__ void k_hist(IfaceDev I, LevelGeo gc, const S *__restrict__ fc, int slot)
{
    using L = Lat<Q>;
    constexpr int D = L::D;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < I.nTF) {
        const long long idx = I.tf_coarse[t];
        const unsigned int kc = I.tf_kc[t];
        for (int i = 0; i < Q; i++) {
            double v = 0.0;
            if ((kc >> i) & 1u) {
                const long long s = shifted_index(gc, idx, -L::c(i, 0), -L::c(i, 1), -L::c(i, 2));
                if (s >= 0) v = (double)St<S>::ld(fc, (long long)i * gc.pitch + s, L::w(i));
            }
            I.hist_f[((long long)slot * Q + i) * I.nTF + t] = v;
        }
    } else if (t < I.nTF + I.nRing) {
        const int r = t - I.nTF;
        const long long idx = I.ring_coarse[r];
        double rho = 0.0, m[3] = {0.0, 0.0, 0.0};
        for (int i = 0; i < Q; i++) {
            const long long s = shifted_index(gc, idx, -L::c(i, 0), -L::c(i, 1), -L::c(i, 2));
            const double v = s >= 0 ? (double)St<S>::ld(fc, (long long)i * gc.pitch + s, L::w(i)) : 0.0;
            rho += v;
            for (int a = 0; a < D; a++) m[a] += L::c(i, a) * v;
        }
        double *h = I.hist_m + (long long)slot * 4 * I.nRing;
        h[r] = rho;
        for (int a = 0; a < 3; a++) h[(long long)(1 + a) * I.nRing + r] = a < D ? m[a] / rho : 0.0;
    }
}

// seed slot 0 from the initial state itself (no streaming)
template <int Q, typename S>
__global__ void k_hist_seed(IfaceDev I, LevelGeo gc, const S *__restrict__ fc)
{
    using L = Lat<Q>;
    constexpr int D = L::D;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < I.nTF) {
        const long long idx = I.tf_coarse[t];
        for (int i = 0; i < Q; i++)
            I.hist_f[(long long)i * I.nTF + t] = (double)St<S>::ld(fc, (long long)i * gc.pitch + idx, L::w(i));
    } else if (t < I.nTF + I.nRing) {
        const int r = t - I.nTF;
        const long long idx = I.ring_coarse[r];
        double rho = 0.0, m[3] = {0.0, 0.0, 0.0};
        for (int i = 0; i < Q; i++) {
            const double v = (double)St<S>::ld(fc, (long long)i * gc.pitch + idx, L::w(i));
            rho += v;
            for (int a = 0; a < D; a++) m[a] += L::c(i, a) * v;
        }
        I.hist_m[r] = rho;
        for (int a = 0; a < 3; a++) I.hist_m[(long long)(1 + a) * I.nRing + r] = a < D ? m[a] / rho : 0.0;
    }
}

// ------------------------------------------------------------------ TF reconstruction
// Newton at TF nodes (Eq. system_fi), fine rebuild of gamma=c populations
// (Eq. rescff), and on sync sub-steps the coarse rebuild of all populations (Eq. rescfc).
template <int Q, typename S>
__global__ void k_recon(IfaceDev I, LevelDev F, LevelDev Cl, const S *__restrict__ ff, TimeW tw, int sync,
                        int *status, int *max_iters)
{
    using L = Lat<Q>;
    constexpr int D = L::D;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= I.nTF) return;
    const long long idx = I.tf_fine[t];
    const unsigned int kf = I.tf_kf[t], gc = I.tf_gc[t];
    double fhat[Q], Gam[Q];
    for (int i = 0; i < Q; i++) {
        if ((gc >> i) & 1u) {
            double s = 0.0;
            for (int k = 0; k < 3; k++)
                if (tw.w[k] != 0.0) s += tw.w[k] * I.hist_f[((long long)tw.slot[k] * Q + i) * I.nTF + t];
            fhat[i] = s;
            Gam[i] = I.R;
        } else {
            double v = 0.0;
            if ((kf >> i) & 1u) {
                const long long s = shifted_index(F.g, idx, -L::c(i, 0), -L::c(i, 1), -L::c(i, 2));
                if (s >= 0) v = (double)St<S>::ld(ff, (long long)i * F.g.pitch + s, L::w(i));
            }
            fhat[i] = v;
            Gam[i] = 1.0;
        }
    }
    double X[4];
    const int it = newton_solve<Q>(fhat, Gam, X);
    if (it < 0) {
        atomicOr(status, ST_NEWTON);
        return;
    }
    atomicMax(max_iters, it);
    const int nif = F.nif;
    for (int i = 0; i < Q; i++) {
        const double fe = feq_one<Q>(i, X[0], X + 1);
        const double v = ((gc >> i) & 1u) ? fe + I.R * (fhat[i] - fe) : fhat[i];
        F.if_pop[(long long)i * nif + t] = v;
        if (sync) Cl.if_pop[(long long)i * Cl.nif + I.tfc_base + t] = fe + (v - fe) / I.R;
    }
    for (int a = 0; a < 4; a++) {
        const double xv = a <= D ? X[a] : 0.0;
        F.if_mac[(long long)a * nif + t] = xv;
        if (sync) Cl.if_mac[(long long)a * Cl.nif + I.tfc_base + t] = xv;
    }
}

// ------------------------------------------------------------------ TF gradients
// Sec. 3.3: centred differences over the coarse stencil (fine nodes two fine cells
// inward, TF neighbours along the interface with their X, coarse ring nodes outward,
// time-interpolated on async sub-steps), rescaled by 1/2 for the fine level.
template <int Q, typename S>
__global__ void k_grad(IfaceDev I, LevelDev F, LevelDev Cl, const S *__restrict__ ff, TimeW tw, int sync)
{
    using L = Lat<Q>;
    constexpr int D = L::D;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= I.nTF) return;
    double rho[3][2], u[3][2][3];
    for (int b = 0; b < D; b++)
        for (int s = 0; s < 2; s++) {
            const int k = t * 2 * D + 2 * b + s;
            const signed char kind = I.tf_rkind[k];
            const long long ref = I.tf_ridx[k];
            double r = 0.0, uu[3] = {0.0, 0.0, 0.0};
            if (kind == RK_TF) {
                r = F.if_mac[ref];
                for (int a = 0; a < D; a++) uu[a] = F.if_mac[(long long)(1 + a) * F.nif + ref];
            } else if (kind == RK_RING) {
                for (int j = 0; j < 3; j++) {
                    if (tw.w[j] == 0.0) continue;
                    const double *h = I.hist_m + (long long)tw.slot[j] * 4 * I.nRing;
                    r += tw.w[j] * h[ref];
                    for (int a = 0; a < D; a++) uu[a] += tw.w[j] * h[(long long)(1 + a) * I.nRing + ref];
                }
            } else {
                double m[3] = {0.0, 0.0, 0.0};
                for (int i = 0; i < Q; i++) {
                    const long long sidx = shifted_index(F.g, ref, -L::c(i, 0), -L::c(i, 1), -L::c(i, 2));
                    const double v = sidx >= 0 ? (double)St<S>::ld(ff, (long long)i * F.g.pitch + sidx, L::w(i)) : 0.0;
                    r += v;
                    for (int a = 0; a < D; a++) m[a] += L::c(i, a) * v;
                }
                for (int a = 0; a < D; a++) uu[a] = m[a] / r;
            }
            rho[b][s] = r;
            for (int a = 0; a < 3; a++) u[b][s][a] = uu[a];
        }
    double Sg[6], Cg[6];
    fd_gradients<D, double>(rho, u, 0.5, Sg, Cg);  // coarse units: neighbours one coarse cell away
    for (int k = 0; k < 6; k++) {
        F.if_S[(long long)k * F.nif + t] = 0.5 * Sg[k];
        F.if_C[(long long)k * F.nif + t] = 0.5 * Cg[k];
        if (sync) {
            Cl.if_S[(long long)k * Cl.nif + I.tfc_base + t] = Sg[k];
            Cl.if_C[(long long)k * Cl.nif + I.tfc_base + t] = Cg[k];
        }
    }
}

// ------------------------------------------------------------------ hanging nodes
// 4-point 1-D Lagrange along the interface (tensor order over odd axes, one-sided
// next to corners) of missing populations, S and C; macros are the moments.
template <int Q, typename S>
__global__ void k_ie(IfaceDev I, LevelDev F, const S *__restrict__ ff)
{
    using L = Lat<Q>;
    constexpr int D = L::D;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= I.nIE) return;
    const long long idx = I.ie_fine[e];
    const unsigned int kf = I.ie_kf[e];
    const int nst = I.ie_nst[e];
    const int row = I.nTF + e;  // table index of this hanging node
    const int nif = F.nif;
    double rho = 0.0, m[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < Q; i++) {
        double v;
        if ((kf >> i) & 1u) {
            const long long s = shifted_index(F.g, idx, -L::c(i, 0), -L::c(i, 1), -L::c(i, 2));
            v = s >= 0 ? (double)St<S>::ld(ff, (long long)i * F.g.pitch + s, L::w(i)) : 0.0;
        } else {
            v = 0.0;
            for (int k = 0; k < nst; k++) v += I.ie_w[e * 16 + k] * F.if_pop[(long long)i * nif + I.ie_st[e * 16 + k]];
        }
        F.if_pop[(long long)i * nif + row] = v;
        rho += v;
        for (int a = 0; a < D; a++) m[a] += L::c(i, a) * v;
    }
    F.if_mac[row] = rho;
    for (int a = 0; a < 3; a++) F.if_mac[(long long)(1 + a) * nif + row] = a < D ? m[a] / rho : 0.0;
    for (int k = 0; k < 6; k++) {
        double s = 0.0, c = 0.0;
        for (int j = 0; j < nst; j++) {
            const int tf = I.ie_st[e * 16 + j];
            s += I.ie_w[e * 16 + j] * F.if_S[(long long)k * nif + tf];
            c += I.ie_w[e * 16 + j] * F.if_C[(long long)k * nif + tf];
        }
        F.if_S[(long long)k * nif + row] = s;
        F.if_C[(long long)k * nif + row] = c;
    }
}

// rho, u of the node at box coordinates (xx, yy, zz) for the shared-memory halo:
// wraps periodic axes, pulls bulk nodes, reads interface nodes from the table;
// returns false (and rho = 1, u = 0) off a non-periodic box or in the hole.
template <int Q, typename S>
__device__ __forceinline__ bool halo_macros(const LevelDev &Lv, const S *__restrict__ fsrc, int xx, int yy, int zz,
                                            typename St<S>::R &hr, typename St<S>::R *hu)
{
    using L = Lat<Q>;
    using R = typename St<S>::R;
    constexpr int D = L::D;
    const LevelGeo &g = Lv.g;
    hr = R(1);
    hu[0] = hu[1] = hu[2] = R(0);
    if (!(wrap_coord(xx, g.n[0], g.per[0]) && wrap_coord(yy, g.n[1], g.per[1]) && wrap_coord(zz, g.n[2], g.per[2])))
        return false;
    const long long hidx = node_index(g, xx, yy, zz);
    const int htag = Lv.tag[hidx];
    if (htag == TAG_BULK) {
        R m[3] = {R(0), R(0), R(0)};
        hr = R(0);
#pragma unroll
        for (int i = 0; i < Q; i++) {
            int sx = xx - L::c(i, 0), sy = yy - L::c(i, 1), sz = zz - L::c(i, 2);
            if (!wrap_coord(sx, g.n[0], g.per[0])) sx = xx;  // bulk sources are nodes: never taken
            if (!wrap_coord(sy, g.n[1], g.per[1])) sy = yy;
            if (!wrap_coord(sz, g.n[2], g.per[2])) sz = zz;
            const R v = St<S>::ld(fsrc, (long long)i * g.pitch + node_index(g, sx, sy, sz), L::w(i));
            hr += v;
#pragma unroll
            for (int a = 0; a < D; a++)
                if (L::c(i, a) != 0) m[a] += R(L::c(i, a)) * v;
        }
#pragma unroll
        for (int a = 0; a < D; a++) hu[a] = m[a] / hr;
        return true;
    }
    if (htag >= 0) {
        hr = (R)Lv.if_mac[htag];
#pragma unroll
        for (int a = 0; a < D; a++) hu[a] = (R)Lv.if_mac[(long long)(1 + a) * Lv.nif + htag];
        return true;
    }
    return false;
}

// ------------------------------------------------------------------ bulk collide-and-stream
// One CTA per tile of TX x TY (x TZ) nodes.  Every node of the tile and of its
// one-node halo pulls its post-stream populations (or reads them from the
// interface table) and stores rho, u in shared memory; then every tile node takes
// centred differences from its neighbours (or the supplied S, C of interface
// nodes) and collides.  Tiles whose tile+2 neighbourhood is all bulk and inside
// the box skip every class test and wrap.
template <int Q, typename S, int TX, int TY, int TZ>
__global__ void __launch_bounds__(TX *TY *TZ) k_bulk(LevelDev Lv, const S *__restrict__ fsrc, S *__restrict__ fdst,
                                                      double sigma, double spsi)
{
    using L = Lat<Q>;
    using R = typename St<S>::R;
    constexpr int D = L::D;
    constexpr int HX = TX + 2, HY = TY + 2, HZ = (D == 3) ? TZ + 2 : 1;
    constexpr int H = HX * HY * HZ;
    constexpr int NT = TX * TY * TZ;
    __shared__ R s_rho[H];
    __shared__ R s_u[D][H];

    const LevelGeo &g = Lv.g;
    const int bx = blockIdx.x % Lv.tiles[0];
    const int by = (blockIdx.x / Lv.tiles[0]) % Lv.tiles[1];
    const int bz = blockIdx.x / (Lv.tiles[0] * Lv.tiles[1]);
    const unsigned char flag = Lv.tile_flag[blockIdx.x];
    if (flag == TILE_SKIP) return;
    const int X0 = bx * TX, Y0 = by * TY, Z0 = bz * (D == 3 ? TZ : 1);
    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = (tid / TX) % TY, tz = tid / (TX * TY);
    const int x = X0 + tx, y = Y0 + ty, z = Z0 + (D == 3 ? tz : 0);
    const long long n01 = (long long)g.n[0] * g.n[1];

    R f[Q];
    R rho = R(0), u[3] = {R(0), R(0), R(0)};
    int tag = TAG_HOLE;
    const bool inside = x < g.n[0] && y < g.n[1] && z < g.n[2];
    const long long idx = (long long)x + (long long)g.n[0] * y + n01 * z;
    const int hself = (tx + 1) + HX * ((ty + 1) + HY * (D == 3 ? tz + 1 : 0));

    if (flag == TILE_FAST) {
        tag = TAG_BULK;
#pragma unroll
        for (int i = 0; i < Q; i++) {
            const long long off = (long long)L::c(i, 0) + (long long)g.n[0] * L::c(i, 1) + n01 * L::c(i, 2);
            f[i] = St<S>::ld(fsrc, (long long)i * g.pitch + idx - off, L::w(i));
        }
    } else if (inside) {
        tag = Lv.tag[idx];
        if (tag == TAG_BULK) {
#pragma unroll
            for (int i = 0; i < Q; i++) {
                int sx = x - L::c(i, 0), sy = y - L::c(i, 1), sz = z - L::c(i, 2);
                if (!wrap_coord(sx, g.n[0], g.per[0])) sx = x;  // bulk sources are nodes: never taken
                if (!wrap_coord(sy, g.n[1], g.per[1])) sy = y;
                if (!wrap_coord(sz, g.n[2], g.per[2])) sz = z;
                f[i] = St<S>::ld(fsrc, (long long)i * g.pitch + node_index(g, sx, sy, sz), L::w(i));
            }
        } else if (tag >= 0) {
#pragma unroll
            for (int i = 0; i < Q; i++) f[i] = (R)Lv.if_pop[(long long)i * Lv.nif + tag];
        }
    }
    if (tag == TAG_BULK) {
        R m[3] = {R(0), R(0), R(0)};
#pragma unroll
        for (int i = 0; i < Q; i++) {
            rho += f[i];
#pragma unroll
            for (int a = 0; a < D; a++)
                if (L::c(i, a) != 0) m[a] += R(L::c(i, a)) * f[i];
        }
#pragma unroll
        for (int a = 0; a < D; a++) u[a] = m[a] / rho;
    } else if (tag >= 0) {
        rho = (R)Lv.if_mac[tag];
#pragma unroll
        for (int a = 0; a < D; a++) u[a] = (R)Lv.if_mac[(long long)(1 + a) * Lv.nif + tag];
    }
    if (flag != TILE_FAST && !inside) {
        // a ragged last tile: on a periodic axis this position is the wrapped node
        R hr, hu[3];
        halo_macros<Q, S>(Lv, fsrc, x, y, z, hr, hu);
        rho = hr;
#pragma unroll
        for (int a = 0; a < D; a++) u[a] = hu[a];
    }
    s_rho[hself] = rho;
#pragma unroll
    for (int a = 0; a < D; a++) s_u[a][hself] = u[a];

    // halo ring
    for (int h = tid; h < H; h += NT) {
        const int hx = h % HX, hy = (h / HX) % HY, hz = h / (HX * HY);
        const bool border = hx == 0 || hx == HX - 1 || hy == 0 || hy == HY - 1 || (D == 3 && (hz == 0 || hz == HZ - 1));
        if (!border) continue;
        int xx = X0 + hx - 1, yy = Y0 + hy - 1, zz = Z0 + (D == 3 ? hz - 1 : 0);
        R hr = R(1), hu[3] = {R(0), R(0), R(0)};
        if (flag == TILE_FAST) {
            const long long hidx = (long long)xx + (long long)g.n[0] * yy + n01 * zz;
            R m[3] = {R(0), R(0), R(0)};
            hr = R(0);
#pragma unroll
            for (int i = 0; i < Q; i++) {
                const long long off = (long long)L::c(i, 0) + (long long)g.n[0] * L::c(i, 1) + n01 * L::c(i, 2);
                const R v = St<S>::ld(fsrc, (long long)i * g.pitch + hidx - off, L::w(i));
                hr += v;
#pragma unroll
                for (int a = 0; a < D; a++)
                    if (L::c(i, a) != 0) m[a] += R(L::c(i, a)) * v;
            }
#pragma unroll
            for (int a = 0; a < D; a++) hu[a] = m[a] / hr;
        } else {
            halo_macros<Q, S>(Lv, fsrc, xx, yy, zz, hr, hu);
        }
        s_rho[h] = hr;
#pragma unroll
        for (int a = 0; a < D; a++) s_u[a][h] = hu[a];
    }
    __syncthreads();
    if (tag == TAG_HOLE || !inside) return;

    R Sv[6], Cv[6];
    if (tag == TAG_BULK) {
        R nr[3][2], nu[3][2][3];
#pragma unroll
        for (int b = 0; b < D; b++)
#pragma unroll
            for (int s = 0; s < 2; s++) {
                const int o = (s == 0 ? 1 : -1);
                const int hh = hself + (b == 0 ? o : (b == 1 ? o * HX : o * HX * HY));
                nr[b][s] = s_rho[hh];
#pragma unroll
                for (int a = 0; a < D; a++) nu[b][s][a] = s_u[a][hh];
                if (D == 2) nu[b][s][2] = R(0);
            }
        fd_gradients<D, R>(nr, nu, R(0.5), Sv, Cv);
    } else {
#pragma unroll
        for (int k = 0; k < 6; k++) {
            Sv[k] = (R)Lv.if_S[(long long)k * Lv.nif + tag];
            Cv[k] = (R)Lv.if_C[(long long)k * Lv.nif + tag];
        }
    }
    hrr_collide<Q, R>(f, rho, u, Sv, Cv, (R)Lv.tau, (R)sigma, (R)spsi);
#pragma unroll
    for (int i = 0; i < Q; i++) St<S>::st(fdst, (long long)i * g.pitch + idx, f[i], L::w(i));
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
    const bool hole = tag[idx] == TAG_HOLE;
    double uu[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < D; a++) uu[a] = u[(long long)a * g.N + idx];
    for (int i = 0; i < Q; i++) {
        const double v = hole ? L::w(i) : feq_one<Q>(i, rho[idx], uu);
        St<S>::st(f0, (long long)i * g.pitch + idx, (typename St<S>::R)v, L::w(i));
        St<S>::st(f1, (long long)i * g.pitch + idx, (typename St<S>::R)v, L::w(i));
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
    const bool hole = tag[idx] == TAG_HOLE;
    double r = 0.0, m[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < Q; i++) {
        const double v = hole ? 0.0 : (double)St<S>::ld(f, (long long)i * g.pitch + idx, L::w(i));
        if (pops) pops[(long long)i * g.N + idx] = v;
        r += v;
        for (int a = 0; a < D; a++) m[a] += L::c(i, a) * v;
    }
    if (rho) rho[idx] = r;
    if (u)
        for (int a = 0; a < D; a++) u[(long long)a * g.N + idx] = hole ? 0.0 : m[a] / r;
}

// Volume-weighted mass and momentum, per-block FP64 partials (deterministic order)
template <int Q, typename S>
__global__ void k_reduce_partial(LevelGeo g, const int *__restrict__ tag, const S *__restrict__ f,
                                 const double *__restrict__ wnode, double *__restrict__ partial, int *status)
{
    using L = Lat<Q>;
    constexpr int D = L::D;
    __shared__ double sh[4][256];
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    bool bad = false;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < g.N;
         idx += (long long)gridDim.x * blockDim.x) {
        if (tag[idx] == TAG_HOLE) continue;
        const double w = wnode[idx];
        for (int i = 0; i < Q; i++) {
            const double v = (double)St<S>::ld(f, (long long)i * g.pitch + idx, L::w(i));
            if (!isfinite(v)) bad = true;
            acc[0] += w * v;
            for (int a = 0; a < D; a++) acc[1 + a] += w * L::c(i, a) * v;
        }
    }
    if (bad) atomicOr(status, ST_NAN);
    for (int k = 0; k < 4; k++) sh[k][threadIdx.x] = acc[k];
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int k = 0; k < 4; k++) sh[k][threadIdx.x] += sh[k][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int k = 0; k < 4; k++) partial[(long long)blockIdx.x * 4 + k] = sh[k][0];
}

__global__ void k_reduce_final(const double *__restrict__ partial, int nblocks, double *__restrict__ out)
{
    __shared__ double sh[4][256];
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
        for (int k = 0; k < 4; k++) acc[k] += partial[(long long)b * 4 + k];
    for (int k = 0; k < 4; k++) sh[k][threadIdx.x] = acc[k];
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int k = 0; k < 4; k++) sh[k][threadIdx.x] += sh[k][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int k = 0; k < 4; k++) out[k] = sh[k][0];
}

}  // namespace lbmg
