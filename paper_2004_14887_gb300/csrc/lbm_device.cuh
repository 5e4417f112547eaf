// Device code of the GB300 direct-coupling multi-level lattice Boltzmann library.
//
// Hot path per level sub-step (Sec. 3.5 of Astoul et al., arXiv 2004.14887):
//   k_recon_hist  Newton at TF nodes (Eqs. system_fi, updated_macro) in the arithmetic
//                 type, fine rebuild of the gamma=c populations (Eq. rescff) and, on
//                 sync sub-steps, coarse rebuild of every population (Eq. rescfc) in
//                 FP64; fused with the history push for the child interface (coarse
//                 post-stream populations at TF nodes and ring macros, Eq. TempInt)
//   k_grad_ie     coarse-stencil S and C = div Psi at TF nodes (Sec. 3.3), x1/2 for
//                 the fine level (Eqs. PijResc, PSIResc); fused with the 4-point 1-D
//                 Lagrange completion of hanging nodes
//   k_bulk2d / k_bulk3d  fused pull-stream + moments (2-D tile or 3-D z-marching
//                 column with staged planes, 1-node halo) + centred finite differences
//                 (Eqs. a1FD_scheme, PSI_FD) + H-RR collision (Eqs. fEq_herm, a12_HRR,
//                 a1Proj, a13RR, LBMscheme_reg, App. A) + store
//   k_batch       all of the above for many D2Q9 hierarchies in one persistent launch
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>
#include <utility>

namespace lbmg {

enum : int { ST_NEWTON = 1, ST_NAN = 2, ST_TIMEOUT = 4 };
enum : signed char { RK_FINE = 0, RK_TF = 1, RK_RING = 2 };
enum : unsigned char { TILE_FAST = 0, TILE_SKIP = 1, TILE_GENERAL = 2 };
enum : int { TAG_BULK = -1, TAG_HOLE = -2 };

// ------------------------------------------------------------------ lattices
template <int Q> struct Lat;

// D2Q9 numbered as the paper's Fig. 1: 0 rest, 1 E, 2 NE, 3 N, 4 NW, 5 W, 6 SW, 7 S, 8 SE
template <> struct Lat<9> {
    static constexpr int D = 2, Q = 9;
    __host__ __device__ static constexpr int c(int i, int a)
    {
        return a == 0 ? ((i == 1 || i == 2 || i == 8) ? 1 : ((i == 4 || i == 5 || i == 6) ? -1 : 0))
                      : (a == 1 ? ((i == 2 || i == 3 || i == 4) ? 1 : ((i == 6 || i == 7 || i == 8) ? -1 : 0)) : 0);
    }
    __host__ __device__ static constexpr double w(int i)
    {
        return i == 0 ? 4.0 / 9.0 : ((i & 1) ? 1.0 / 9.0 : 1.0 / 36.0);
    }
};

// D3Q19 in the paper's groups: 0 rest, 1-6 axes, 7-18 face diagonals (opposites adjacent)
template <> struct Lat<19> {
    static constexpr int D = 3, Q = 19;
    __host__ __device__ static constexpr int c(int i, int a)
    {
        constexpr int t[19][3] = {{0, 0, 0},  {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},   {0, -1, 0},
                                  {0, 0, 1},  {0, 0, -1}, {1, 1, 0},  {-1, -1, 0}, {1, -1, 0},
                                  {-1, 1, 0}, {1, 0, 1},  {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
                                  {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
        return t[i][a];
    }
    __host__ __device__ static constexpr double w(int i)
    {
        return i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
    }
};

// compile-time loop: f(std::integral_constant<int, i>) for i = 0..N-1, so that every
// lattice constant used inside is a constant expression
template <typename F, int... I>
__host__ __device__ __forceinline__ void static_for_impl(F &&f, std::integer_sequence<int, I...>)
{
    (f(std::integral_constant<int, I>{}), ...);
}
template <int N, typename F>
__host__ __device__ __forceinline__ void static_for(F &&f)
{
    static_for_impl(f, std::make_integer_sequence<int, N>{});
}

// symmetric tensors: 0 xx, 1 yy, 2 zz, 3 xy, 4 xz, 5 yz
__host__ __device__ constexpr int sym_index(int a, int b)
{
    return a == b ? a : ((a + b == 1) ? 3 : ((a + b == 2) ? 4 : 5));
}

// ------------------------------------------------------------------ storage
template <typename S> struct St;
template <> struct St<double> {
    using R = double;
    __device__ static __forceinline__ double ld(const double *p, long long k, double) { return p[k]; }
    __device__ static __forceinline__ void st(double *p, long long k, double v, double) { p[k] = v; }
};
template <> struct St<float> {
    using R = float;
    __device__ static __forceinline__ float ld(const float *p, long long k, float) { return p[k]; }
    __device__ static __forceinline__ void st(float *p, long long k, float v, float) { p[k] = v; }
};
// IEEE half storing the deviation f_i - w_i from rest equilibrium, FP32 arithmetic
template <> struct St<__half> {
    using R = float;
    __device__ static __forceinline__ float ld(const __half *p, long long k, float w)
    {
        return __half2float(p[k]) + w;
    }
    __device__ static __forceinline__ void st(__half *p, long long k, float v, float w)
    {
        p[k] = __float2half_rn(v - w);
    }
};

// correctly rounded reciprocal (IEEE round-to-nearest in both types)
__device__ __forceinline__ float recip(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }

// ------------------------------------------------------------------ device views
struct LevelGeo {
    int n[3];
    int per[3];
    int px;           // row pitch in slots: n[0] padded to a multiple of 8
    float shift[19];  // FP16-shifted storage keeps f_i - shift[i] (f_i^eq(1, u_shift))
    long long N;      // box nodes n[0] n[1] n[2] (dense order of the host arrays)
    long long NS;     // slots px n[1] n[2] of the tag map and population planes
    long long pitch;  // elements between population planes (>= NS)
};

struct LevelDev {
    LevelGeo g;
    void *f[2];              // population buffers (storage type), [Q][pitch]
    const int *tag;          // per node: TAG_BULK, TAG_HOLE or interface-table index
    int tiles[3];
    void *if_pop;            // interface table (type R): completed post-stream populations [Q][nif]
    void *if_mac;            // rho, ux, uy, uz [4][nif]
    void *if_S;              // strain rate [6][nif]
    void *if_C;              // C_ab = sum_g d_g Psi_abg [6][nif]
    int nif;
    double tau;
    // geometric tile classification (see tile_class)
    int fast_lo[3], fast_hi[3];  // tile grown by 2 must stay in [fast_lo, fast_hi]
    int has_child;
    int child_lo[3], child_hi[3], child_per[3];  // closed child box in this level's box coordinates
    const unsigned char *tile_flags;  // 2-D: per-tile class (staircase regions), else NULL (geometric rule)
    // collision parameters of the level in both arithmetic types (batched launches read them here)
    double om, sigma, spsi;
    float tauf, omf, sigmaf, spsif;
    // hanging nodes of this level: table rows [ie_base, ie_base + n_ie), TF stencils
    int ie_base, n_ie;
    const int *ie_nst;
    const int *ie_st;
    const void *ie_w;  // [n_ie][16] stencil weights in the arithmetic type
    // FP16-shifted storage (D3Q19 bulk kernel): moments of the shift s_i (sum s, sum c_a
    // s, sum c_a c_b s in the order xx yy zz xy xz yz), and per opposite pair (i odd,
    // opp(i) = i + 1) s_i = w_i (she_i + sho_i), s_opp(i) = w_i (she_i - sho_i); she_0 =
    // s_0 / w_0
    float smom[10];
    float she[19], sho[19];
};

// wrap (periodic) or reject a coordinate; returns false outside a non-periodic box
__device__ __forceinline__ bool wrap_coord(int &v, int n, int per)
{
    if (v >= 0 && v < n) return true;
    if (!per) return false;
    v %= n;  // any distance: ragged tiles may sit more than one period past a short axis
    if (v < 0) v += n;
    return true;
}

// slot of the node with dense index idx (x fastest over n[0], n[1], n[2])
__device__ __forceinline__ long long dense_to_slot(const LevelGeo &g, long long idx)
{
    const long long x = idx % g.n[0], yz = idx / g.n[0];
    return x + (long long)g.px * yz;
}

// ------------------------------------------------------------------ H-RR physics
// Third-moment deviation Psi_abg of App. A (Eq. Psi), reading: D2Q9 keeps only the
// aaa components, D3Q19 keeps aaa, aab (= rho u_b u_g^2 / 2) and xyz.
template <int D, typename R>
__device__ __forceinline__ void psi_components(R rho, const R *u, R *P)
{
    // P: 0 xxx 1 yyy 2 zzz 3 xxy 4 xxz 5 xyy 6 xzz 7 yyz 8 yzz 9 xyz
    P[0] = rho * u[0] * u[0] * u[0];
    P[1] = rho * u[1] * u[1] * u[1];
    if (D == 3) {
        P[2] = rho * u[2] * u[2] * u[2];
        P[3] = R(0.5) * rho * u[1] * u[2] * u[2];  // xxy: single y, third z
        P[4] = R(0.5) * rho * u[2] * u[1] * u[1];  // xxz: single z, third y
        P[5] = R(0.5) * rho * u[0] * u[2] * u[2];  // xyy: single x, third z
        P[6] = R(0.5) * rho * u[0] * u[1] * u[1];  // xzz: single x, third y
        P[7] = R(0.5) * rho * u[2] * u[0] * u[0];  // yyz: single z, third x
        P[8] = R(0.5) * rho * u[1] * u[0] * u[0];  // yzz: single y, third x
        P[9] = rho * u[0] * u[1] * u[2];
    }
}

// Centred differences from the macros of the 2D axis neighbours (m[b][0] at +e_b,
// m[b][1] at -e_b), half-width h nodes: S_ab and C_ab = sum_g d_g Psi_abg.
template <int D, typename R>
__device__ __forceinline__ void fd_gradients(const R (&rho)[3][2], const R (&u)[3][2][3], R inv2h, R *S, R *C)
{
    R du[3][3];  // du[b][a] = d_b u_a
#pragma unroll
    for (int b = 0; b < D; b++)
#pragma unroll
        for (int a = 0; a < D; a++) du[b][a] = (u[b][0][a] - u[b][1][a]) * inv2h;
    R dP[3][10];  // dP[g][k] = d_g P_k
#pragma unroll
    for (int g = 0; g < D; g++) {
        R Pp[10], Pm[10];
        psi_components<D, R>(rho[g][0], u[g][0], Pp);
        psi_components<D, R>(rho[g][1], u[g][1], Pm);
#pragma unroll
        for (int k = 0; k < (D == 3 ? 10 : 2); k++) dP[g][k] = (Pp[k] - Pm[k]) * inv2h;
    }
    S[0] = du[0][0];
    S[1] = du[1][1];
    S[3] = R(0.5) * (du[1][0] + du[0][1]);
    if (D == 2) {
        S[2] = S[4] = S[5] = R(0);
        C[0] = dP[0][0];
        C[1] = dP[1][1];
        C[2] = C[3] = C[4] = C[5] = R(0);
    } else {
        S[2] = du[2][2];
        S[4] = R(0.5) * (du[2][0] + du[0][2]);
        S[5] = R(0.5) * (du[2][1] + du[1][2]);
        C[0] = dP[0][0] + dP[1][3] + dP[2][4];  // d_x Pxxx + d_y Pxxy + d_z Pxxz
        C[1] = dP[0][5] + dP[1][1] + dP[2][7];  // d_x Pxyy + d_y Pyyy + d_z Pyyz
        C[2] = dP[0][6] + dP[1][8] + dP[2][2];  // d_x Pxzz + d_y Pyzz + d_z Pzzz
        C[3] = dP[0][3] + dP[1][5] + dP[2][9];  // d_x Pxxy + d_y Pxyy + d_z Pxyz
        C[4] = dP[0][4] + dP[1][9] + dP[2][6];  // d_x Pxxz + d_y Pxyz + d_z Pxzz
        C[5] = dP[0][9] + dP[1][7] + dP[2][8];  // d_x Pxyz + d_y Pyyz + d_z Pyzz
    }
}

// H-RR collision of one node, Eq. (LBMscheme_reg), in the compact Hermite form
//   f_i = w_i [ rho (1 + c.u/cs2) + H2_i:B/(2cs2^2) + sum_{a!=b} H3_i,aab T_ab/(2cs2^3) ]
// with B = rho uu + (1-1/tau) a1 + (s/2) C and T_ab = rho u_a^2 u_b + (1-1/tau) a1_aab,
// which is f0 + (1-1/tau) f1_reg + psi/2 term by term (om = 1 - 1/tau).  a1 follows Eq. (a12_HRR):
// a1^PR = sum_i H2_i (f_i - f0_i + psi_i/2) = Pi - cs2 sum(f) I - rho uu + (s/2) C
// (Hermite orthogonality), a1^FD = -2 tau rho cs2 S.
template <int Q, typename R>
__device__ __forceinline__ void hrr_collide(R (&f)[Q], R rho, const R *u, const R *S, const R *C, R tau, R om,
                                            R sigma, R spsi)
{
    using L = Lat<Q>;
    constexpr int D = L::D;
    const R cs2 = R(1) / R(3);
    R Pi[6] = {0, 0, 0, 0, 0, 0};
    R fsum = R(0);
    static_for<Q>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        fsum += f[i];
        static_for<D>([&](auto ac) {
            constexpr int a = decltype(ac)::value;
            static_for<D>([&](auto bc) {
                constexpr int b = decltype(bc)::value;
                constexpr int p = L::c(i, a) * L::c(i, b);
                if constexpr (b >= a && p != 0) {
                    if constexpr (p > 0) Pi[sym_index(a, b)] += f[i];
                    else Pi[sym_index(a, b)] -= f[i];
                }
            });
        });
    });
    const R kfd = R(-2) * tau * rho * cs2;
    R B[6], A[6];
#pragma unroll
    for (int a = 0; a < D; a++)
#pragma unroll
        for (int b = a; b < D; b++) {
            const int k = sym_index(a, b);
            const R ruu = rho * u[a] * u[b];
            R apr = Pi[k] - ruu + R(0.5) * spsi * C[k];
            if (a == b) apr -= cs2 * fsum;
            A[k] = sigma * apr + (R(1) - sigma) * kfd * S[k];
            B[k] = ruu + om * A[k] + R(0.5) * spsi * C[k];
        }
    R T[3][3];
#pragma unroll
    for (int a = 0; a < D; a++)
#pragma unroll
        for (int b = 0; b < D; b++)
            if (a != b) T[a][b] = rho * u[a] * u[a] * u[b] + om * (R(2) * u[a] * A[sym_index(a, b)] + u[b] * A[sym_index(a, a)]);
    R trB = R(0);
#pragma unroll
    for (int a = 0; a < D; a++) trB += B[sym_index(a, a)];
    const R base = rho, r3 = R(3) * rho, ctr = cs2 * trB;
    static_for<Q>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        R cu = R(0), h2 = -ctr, h3 = R(0);
        static_for<D>([&](auto ac) {
            constexpr int a = decltype(ac)::value;
            constexpr int ca = L::c(i, a);
            if constexpr (ca != 0) {
                if constexpr (ca > 0) cu += u[a];
                else cu -= u[a];
                h2 += B[sym_index(a, a)];
            }
            static_for<D>([&](auto bc) {
                constexpr int b = decltype(bc)::value;
                constexpr int cb = L::c(i, b);
                if constexpr (b > a && ca * cb != 0) h2 += R(2 * ca * cb) * B[sym_index(a, b)];
                // H3_aab = (c_a^2 - cs2) c_b, for a != b and c_b != 0
                if constexpr (a != b && cb != 0) {
                    constexpr double k3 = ((double)(ca * ca) - 1.0 / 3.0) * cb;
                    h3 += R(k3) * T[a][b];
                }
            });
        });
        f[i] = R(L::w(i)) * (base + r3 * cu + R(4.5) * h2 + R(13.5) * h3);
    });
}

// Equilibrium of Eq. (fEq_herm) of population i
template <int Q>
__host__ __device__ __forceinline__ double feq_one(int i, double rho, const double *u)
{
    using L = Lat<Q>;
    constexpr int D = L::D;
    const double cs2 = 1.0 / 3.0;
    double cu = 0.0, uu = 0.0, h3 = 0.0;
    for (int a = 0; a < D; a++) {
        cu += L::c(i, a) * u[a];
        uu += u[a] * u[a];
    }
    for (int a = 0; a < D; a++)
        for (int b = 0; b < D; b++)
            if (a != b) h3 += (L::c(i, a) * L::c(i, a) - cs2) * L::c(i, b) * u[a] * u[a] * u[b];
    return L::w(i) * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu + 13.5 * h3);
}

}  // namespace lbmg
