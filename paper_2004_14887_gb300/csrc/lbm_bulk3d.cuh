// D3Q19 bulk collide-and-stream: one CTA per TX x TY column of nodes marching in z
// over a chunk of planes, each plane's incoming populations staged in shared memory
// by bulk tensor copies (Sec. 2 H-RR collision with the centred differences of
// Eqs. (a1FD_scheme) and (PSI_FD); Sec. 3.5 steps 2h / 3g).
//
// Work per node and plane, in the order of one loop iteration (plane p):
//   pull     the node's 19 post-stream populations from the stage; their moments
//            (sum f, sum c f, sum c c f) in pair sums f_i +- f_opp(i); FP16-shifted
//            storage sums the stored deviations and adds the moments of the shift
//   ring     u and the nine Psi components of App. A that in-plane neighbours
//            difference (all but Psi_zzz) into a two-slot ring in shared memory, once
//            per node (the column's one-node halo included); u and the six Psi
//            components that z differences need stay in registers (this plane and
//            the two before)
//   collide  plane p - 1: S and C from the in-plane differences taken one plane
//            earlier and the z differences of the register copies; H-RR from the
//            eight carried moments (rho, sum f, Pi) in the pair form of Eq.
//            (LBMscheme_reg): f_i, f_opp(i) = w_i (E +- O), E even and O odd in c_i
//   in-plane differences of plane p from the ring (128-bit shared loads)
// Interface nodes take populations, macros, S and C from the level's interface table
// (the S and C rows of hanging nodes are interpolated from the TF rows beforehand).
#pragma once

#include "lbm_kernels.cuh"

namespace lbmg {

// arrive on an mbarrier (release at CTA scope: the thread's earlier shared-memory
// writes are visible to threads whose wait on the phase completes)
__device__ __forceinline__ void mbar_arrive(unsigned long long *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tma::saddr(bar)) : "memory");
}

// populations of D3Q19 with c_z = +1 and c_z = -1, as bit masks
constexpr unsigned cz_mask(int sign)
{
    unsigned m = 0;
    for (int i = 0; i < 19; i++)
        if (Lat<19>::c(i, 2) == sign) m |= 1u << i;
    return m;
}
constexpr unsigned kCzPlus = cz_mask(1), kCzMinus = cz_mask(-1);

// Runs of consecutive populations (storage order) with the same c_z: the populations of a
// run stream from the same plane, so one tensor copy of depth 1, 2, 4 or 5 in the
// population axis moves the whole run.  D3Q19: 0-4, 5, 6, 7-10, 11, 12-13, 14-15, 16-17, 18.
constexpr int kRuns = 9;
constexpr int run_start(int j)
{
    int r = 0, i = 0;
    while (r < j) {
        int e = i + 1;
        while (e < 19 && Lat<19>::c(e, 2) == Lat<19>::c(i, 2)) e++;
        i = e;
        r++;
    }
    return i;
}
constexpr int run_len(int j)
{
    const int i = run_start(j);
    int e = i + 1;
    while (e < 19 && Lat<19>::c(e, 2) == Lat<19>::c(i, 2)) e++;
    return e - i;
}
static_assert(run_start(kRuns) == 19, "nine runs cover the 19 populations");
// tensor map of a run: box depth 1, 2, 4 or 5 populations
constexpr int depth_map(int len) { return len == 1 ? 0 : (len == 2 ? 1 : (len == 4 ? 2 : 3)); }
constexpr int kDepths[4] = {1, 2, 4, 5};
struct alignas(64) TMaps {
    CUtensorMap m[4];  // boxes of 1, 2, 4 and 5 populations
};

// shapes of the 3-D staged kernel for storage S and a TX x TY column
template <int Q, typename S, int TX, int TY>
struct Stage3 {
    using R = typename St<S>::R;
    static constexpr int XA = 16 / (int)sizeof(S);   // x reach of the box below X0 (one 16-byte step)
    static constexpr int BW = TX + 2 * XA;           // box: x in [X0-XA, X0+TX+XA), y in [Y0-2, Y0+TY+2)
    static constexpr int BH = TY + 4;
    static constexpr int BOX = BW * BH;               // elements of one population's box
    static constexpr int HX = TX + 2, HY = TY + 2, HP = HX * HY;  // macro tile with its one-node halo
    static constexpr int NV = 12;                    // ring values per node: u (3), 9 Psi components
    static constexpr int NRING = 2;                  // ring slots: plane p (written) and p - 1 (read)
    static constexpr size_t stage_bytes = (size_t)Q * BOX * sizeof(S);
    static constexpr size_t ring_bytes = (size_t)NRING * HP * NV * sizeof(R);
    static constexpr size_t smem_bytes = 128 + 2 * stage_bytes + ring_bytes + 32;  // +128: alignment of the base
    static_assert((BOX * sizeof(S)) % 128 == 0, "population boxes stay 128-byte aligned");
    static_assert(ring_bytes % 16 == 0, "16-byte aligned ring and barriers");
    static_assert(BW <= 256 && BH <= 256, "tensor box limits");
};

// ring values of a node: 0-2 u, 3 Psi_xxx, 4 Psi_yyy, 5 Psi_xxy, 6 Psi_xxz, 7 Psi_xyy,
// 8 Psi_xzz, 9 Psi_yzz, 10 Psi_yyz, 11 Psi_xyz; z values (registers): 0-2 u, 3 Psi_zzz,
// 4 Psi_xxz, 5 Psi_yyz, 6 Psi_xyz, 7 Psi_xzz, 8 Psi_yzz
enum : int { RV_PXXX = 3, RV_PYYY, RV_PXXY, RV_PXXZ, RV_PXYY, RV_PXZZ, RV_PYZZ, RV_PYYZ, RV_PXYZ };
enum : int { ZV_PZZZ = 3, ZV_PXXZ, ZV_PYYZ, ZV_PXYZ, ZV_PXZZ, ZV_PYZZ };

// Psi components of App. A (Eq. Psi) with the D3Q19 reading: Psi_aaa = rho u_a^3,
// Psi_aab = rho u_b u_g^2 / 2 (g the third axis), Psi_xyz = rho u_x u_y u_z; written to
// the ring values rv and the z values zv
template <typename R>
__device__ __forceinline__ void psi_ring(R rho, const R *u, R (&rv)[12], R (&zv)[9])
{
    const R xx = u[0] * u[0], yy = u[1] * u[1], zz = u[2] * u[2];
    const R jx = rho * u[0], jy = rho * u[1], jz = rho * u[2];  // rho u_a
    const R hx = R(0.5) * jx, hy = R(0.5) * jy, hz = R(0.5) * jz;
    rv[0] = zv[0] = u[0];
    rv[1] = zv[1] = u[1];
    rv[2] = zv[2] = u[2];
    rv[RV_PXXX] = jx * xx;
    rv[RV_PYYY] = jy * yy;
    zv[ZV_PZZZ] = jz * zz;
    rv[RV_PXXY] = hy * zz;               // xxy: single y, third z
    rv[RV_PXXZ] = zv[ZV_PXXZ] = hz * yy;  // xxz: single z, third y
    rv[RV_PXYY] = hx * zz;               // xyy: single x, third z
    rv[RV_PXZZ] = zv[ZV_PXZZ] = hx * yy;  // xzz: single x, third y
    rv[RV_PYYZ] = zv[ZV_PYYZ] = hz * xx;  // yyz: single z, third x
    rv[RV_PYZZ] = zv[ZV_PYZZ] = hy * xx;  // yzz: single y, third x
    rv[RV_PXYZ] = zv[ZV_PXYZ] = jx * u[1] * u[2];
}

// 12 ring values of a node with 16-byte shared-memory accesses
template <typename R>
__device__ __forceinline__ void ring_store(R *p, const R (&v)[12])
{
    if constexpr (sizeof(R) == 4) {
        float4 *q = reinterpret_cast<float4 *>(p);
        q[0] = make_float4(v[0], v[1], v[2], v[3]);
        q[1] = make_float4(v[4], v[5], v[6], v[7]);
        q[2] = make_float4(v[8], v[9], v[10], v[11]);
    } else {
        double2 *q = reinterpret_cast<double2 *>(p);
#pragma unroll
        for (int k = 0; k < 6; k++) q[k] = make_double2(v[2 * k], v[2 * k + 1]);
    }
}
template <typename R>
__device__ __forceinline__ void ring_load(const R *p, R (&v)[12])
{
    if constexpr (sizeof(R) == 4) {
        const float4 *q = reinterpret_cast<const float4 *>(p);
        const float4 a = q[0], b = q[1], c = q[2];
        v[0] = a.x, v[1] = a.y, v[2] = a.z, v[3] = a.w;
        v[4] = b.x, v[5] = b.y, v[6] = b.z, v[7] = b.w;
        v[8] = c.x, v[9] = c.y, v[10] = c.z, v[11] = c.w;
    } else {
        const double2 *q = reinterpret_cast<const double2 *>(p);
#pragma unroll
        for (int k = 0; k < 6; k++) {
            const double2 a = q[k];
            v[2 * k] = a.x, v[2 * k + 1] = a.y;
        }
    }
}

// stored value of a population in the arithmetic type, without the FP16 shift
template <typename S>
__device__ __forceinline__ typename St<S>::R raw(S v)
{
    if constexpr (std::is_same<S, __half>::value) return __half2float(v);
    else return v;
}

// Moments of 19 population values (D3Q19) from the pair sums s_i = f_i + f_opp(i) and
// differences d_i = f_i - f_opp(i) (i odd), in short independent chains: m[0] = sum f,
// m[1..3] = sum c_a f, m[4..9] = sum c_a c_b f (xx yy zz xy xz yz).  With ONLY_J the
// second moments are skipped (halo nodes need rho and u only).
template <typename R, bool ONLY_J = false>
__device__ __forceinline__ void pair_moments19(const R (&v)[19], R (&m)[10])
{
    // pairs: 1/2 +-x, 3/4 +-y, 5/6 +-z, 7/8 +-(1,1,0), 9/10 +-(1,-1,0), 11/12 +-(1,0,1),
    // 13/14 +-(1,0,-1), 15/16 +-(0,1,1), 17/18 +-(0,1,-1)
    const R s1 = v[1] + v[2], s3 = v[3] + v[4], s5 = v[5] + v[6], s7 = v[7] + v[8], s9 = v[9] + v[10];
    const R s11 = v[11] + v[12], s13 = v[13] + v[14], s15 = v[15] + v[16], s17 = v[17] + v[18];
    const R d1 = v[1] - v[2], d3 = v[3] - v[4], d5 = v[5] - v[6], d7 = v[7] - v[8], d9 = v[9] - v[10];
    const R d11 = v[11] - v[12], d13 = v[13] - v[14], d15 = v[15] - v[16], d17 = v[17] - v[18];
    const R qxy = s7 + s9, qxz = s11 + s13, qyz = s15 + s17;
    m[0] = ((v[0] + s1) + (s3 + s5)) + ((qxy + qxz) + qyz);
    m[1] = (d1 + (d7 + d9)) + (d11 + d13);
    m[2] = (d3 + (d7 - d9)) + (d15 + d17);
    m[3] = (d5 + (d11 - d13)) + (d15 - d17);
    if constexpr (!ONLY_J) {
        m[4] = (s1 + qxy) + qxz;
        m[5] = (s3 + qxy) + qyz;
        m[6] = (s5 + qxz) + qyz;
        m[7] = s7 - s9;
        m[8] = s11 - s13;
        m[9] = s15 - s17;
    }
}

// H-RR post-collision populations of one node from its moments, Eq. (LBMscheme_reg) in
// the compact Hermite form of hrr_collide: f_i = w_i [rho (1 + c_i.u/cs2) + H2_i:B /
// (2 cs2^2) + sum_{a!=b} H3_i,aab T_ab / (2 cs2^3)] with B = rho uu + om a1 + (s/2) C and
// T_ab = rho u_a^2 u_b + om a1_aab (Eqs. a12_HRR, a13RR, App. A), evaluated per opposite
// pair as f_i = w_i (E + O), f_opp(i) = w_i (E - O), with the even part E = rho +
// (9/2) H2_i:B and the odd part O = 3 rho c_i.u + (27/2) sum_{a!=b} H3_i,aab T_ab.  The
// third-order sum of a diagonal pair in the plane of axes a, b is c_a V_a^b + c_b V_b^a
// with V_b^a = T_ab + W_b, where W_b = -(1/3) sum_{a!=b} T_ab is the whole sum of the
// axis population along +b.  Pq is sum c c f of the pre-collision populations with
// cs2 sum f taken off its diagonal.  With SHIFT the values returned are f_i - s_i with
// s_i = w_i (she_i + sho_i), s_opp(i) = w_i (she_i - sho_i); PLAIN: the shift of a
// fluid at rest, s_i = w_i (she_i = 1, sho_i = 0), folded into the constants.
template <typename R, bool SHIFT, bool PLAIN, typename Put>
__device__ __forceinline__ void hrr_pairs19(R rho, const R *u, const R *Pq, const R *S, const R *C, R tau, R om,
                                            R sigma, R spsi, const float *she, const float *sho, Put &&put)
{
    using L = Lat<19>;
    const R cs2 = R(1) / R(3);
    const R kfd = R(-2) * tau * rho * cs2;
    const R hs = R(0.5) * spsi;
    const R sg1 = R(1) - sigma;
    R A[6], B[6], ruu[6];
#pragma unroll
    for (int k = 0; k < 6; k++) {
        const int a = k < 3 ? k : (k == 5 ? 1 : 0), b = k < 3 ? k : (k == 3 ? 1 : 2);
        ruu[k] = rho * u[a] * u[b];
        const R hc = hs * C[k];
        const R apr = Pq[k] - ruu[k] + hc;  // a1^PR of Eq. (a1Proj): Pi - cs2 sum f I - rho uu + psi part
        A[k] = sigma * apr + sg1 * kfd * S[k];
        B[k] = ruu[k] + om * A[k] + hc;
    }
    // T_ab = rho u_a^2 u_b + om (2 u_a A_ab + u_b A_aa)
    R T[3][3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const R ua2 = R(2) * u[a];
#pragma unroll
        for (int b = 0; b < 3; b++)
            if (a != b) T[a][b] = ruu[a] * u[b] + om * (ua2 * A[sym_index(a, b)] + u[b] * A[a]);
    }
    const R third = R(1) / R(3);
    const R W[3] = {-third * (T[1][0] + T[2][0]), -third * (T[0][1] + T[2][1]), -third * (T[0][2] + T[1][2])};
    const R ctr = cs2 * (B[0] + B[1] + B[2]);
    const R r3 = R(3) * rho;
    // one output pair: population i (compile time) with cu = c_i.u, h2 = H2_i:B and h3 =
    // sum_{a!=b} H3_i,aab T_ab; its opposite is i + 1
    auto out = [&](auto ic, R cu, R h2, R h3) {
        constexpr int i = decltype(ic)::value;
        R e = rho + R(4.5) * h2;
        R o = r3 * cu + R(13.5) * h3;
        if constexpr (SHIFT && PLAIN) {
            e -= R(1);
        } else if constexpr (SHIFT) {
            e -= R(she[i]);
            o -= R(sho[i]);
        }
        const R w = R(L::w(i)), we = w * e;
        put(std::integral_constant<int, i>{}, we + w * o);
        put(std::integral_constant<int, i + 1>{}, we - w * o);
    };
    {
        const R e = rho - R(4.5) * ctr;  // rest population: E = rho - 9/2 cs2 tr B, O = 0
        if constexpr (SHIFT) put(std::integral_constant<int, 0>{}, R(L::w(0)) * (e - (PLAIN ? R(1) : R(she[0]))));
        else put(std::integral_constant<int, 0>{}, R(L::w(0)) * e);
    }
    out(std::integral_constant<int, 1>{}, u[0], B[0] - ctr, W[0]);
    out(std::integral_constant<int, 3>{}, u[1], B[1] - ctr, W[1]);
    out(std::integral_constant<int, 5>{}, u[2], B[2] - ctr, W[2]);
    {
        const R t = (B[0] + B[1]) - ctr, Vxy = T[1][0] + W[0], Vyx = T[0][1] + W[1];
        out(std::integral_constant<int, 7>{}, u[0] + u[1], t + R(2) * B[3], Vxy + Vyx);
        out(std::integral_constant<int, 9>{}, u[0] - u[1], t - R(2) * B[3], Vxy - Vyx);
    }
    {
        const R t = (B[0] + B[2]) - ctr, Vxz = T[2][0] + W[0], Vzx = T[0][2] + W[2];
        out(std::integral_constant<int, 11>{}, u[0] + u[2], t + R(2) * B[4], Vxz + Vzx);
        out(std::integral_constant<int, 13>{}, u[0] - u[2], t - R(2) * B[4], Vxz - Vzx);
    }
    {
        const R t = (B[1] + B[2]) - ctr, Vyz = T[2][1] + W[1], Vzy = T[1][2] + W[2];
        out(std::integral_constant<int, 15>{}, u[1] + u[2], t + R(2) * B[5], Vyz + Vzy);
        out(std::integral_constant<int, 17>{}, u[1] - u[2], t - R(2) * B[5], Vyz - Vzy);
    }
}

// 3-D z-marching bulk kernel.  One CTA per TX x TY column of nodes and chunk of planes
// [zb, ze).  For each plane p the populations that stream into it (population i from
// plane p - c_iz, over the column grown by XA nodes in x and 2 in y) arrive in a
// shared-memory stage by bulk tensor copies (or, for a column that meets a periodic
// seam in x or y, by 16-byte or element copies with wrapped coordinates), one plane
// ahead of the plane being used, in a ring of two stages with an mbarrier each.  Waits
// are bounded: on time-out the kernel sets ST_TIMEOUT, waits (bounded) for its copies
// in flight and returns.  withhold_block / withhold_k (test hook, -1: none): the block
// with that linear index does not issue the copies of its k-th stage, so its wait for
// them runs out.  PLAIN (FP16 storage with u_shift = 0): the shift's moments and pair
// constants are compile-time values; the results are the same bits as with the
// general shift tables, whose entries are then exactly 1, 0 and 1/3 in FP32.
template <int Q, typename S, int TX, int TY, bool PLAIN = false>
__global__ void __launch_bounds__(TX *TY, sizeof(S) == 8 ? 1 : 2)
    k_bulk3d(const __grid_constant__ TMaps tmaps, const __grid_constant__ LevelDev Lv, const S *__restrict__ fsrc, S *__restrict__ fdst,
             typename St<S>::R tau, typename St<S>::R om, typename St<S>::R sigma, typename St<S>::R spsi, int zc,
             int *status, unsigned long long limit_ns, int withhold_block, int withhold_k)
{
    pdl_enter();
    using L = Lat<Q>;
    using G = Stage3<Q, S, TX, TY>;
    using R = typename St<S>::R;
    constexpr bool SHIFT = std::is_same<S, __half>::value;
    static_assert(Q == 19, "D3Q19 kernel");
    constexpr int XA = G::XA, BW = G::BW, BOX = G::BOX, HX = G::HX, HP = G::HP, NV = G::NV, NT = TX * TY;
    constexpr int NB = 2 * TX + 2 * TY;  // halo nodes that neighbours read (corners are not)
    static_assert(NB <= NT, "one halo node per thread at most");
    extern __shared__ unsigned char smem_raw[];
    unsigned char *base = smem_raw + ((128u - (tma::saddr(smem_raw) & 127u)) & 127u);  // 128-byte aligned stages
    auto stage = [&](int s) { return (S *)(base + (size_t)s * G::stage_bytes); };
    R *ring = (R *)(base + 2 * G::stage_bytes);  // [NRING][HP][NV]
    unsigned long long *bar = (unsigned long long *)(base + 2 * G::stage_bytes + G::ring_bytes);

    const LevelGeo &g = Lv.g;
    const int X0 = blockIdx.x * TX, Y0 = blockIdx.y * TY;
    const int zb = blockIdx.z * zc, ze = min(zb + zc, g.n[2]);
    if (zb >= ze) return;
    const int blin = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;
    const int x = X0 + tx, y = Y0 + ty;
    const bool in_xy = x < g.n[0] && y < g.n[1];
    const int hs = (tx + 1) + HX * (ty + 1);
    // the halo nodes (the four corners are never read) go to the first threads, so that
    // they fill whole warps: NB / 32 warps pull a halo node besides their own node and
    // arrive at the ring's split barrier later than the others, which spend that time
    // on the collision of the plane below
    constexpr int NW = NT / 32;
    const int hn = tid;
    int hb = -1, hx = 0, hy = 0;
    if (hn < NB) {
        if (hn < TX) {
            hx = hn + 1;
            hy = 0;
        } else if (hn < 2 * TX) {
            hx = hn - TX + 1;
            hy = TY + 1;
        } else {
            const int b = hn - 2 * TX;
            hy = 1 + (b >> 1);
            hx = (b & 1) ? HX - 1 : 0;
        }
        hb = hx + HX * hy;
    }
    // own node and halo node in box coordinates (bx, by) of a stage
    const int own_b = (ty + 2) * BW + (tx + XA);
    const int halo_b = (hy + 1) * BW + (hx - 1 + XA);
    const int n01 = g.px * g.n[1];
    const long long pitch = g.pitch;
    // a column whose stage would cross a periodic seam in x or y is filled by plain loads
    const bool seam = (g.per[0] && (X0 - 2 < 0 || X0 + TX + 1 > g.n[0] - 1)) ||
                      (g.per[1] && (Y0 - 2 < 0 || Y0 + TY + 1 > g.n[1] - 1));
    // seam stages in 16-byte chunks when a periodic x extent is whole chunks, else by
    // elements; both asynchronous except element copies of 2-byte storage
    const bool chunked = !g.per[0] || g.n[0] % (16 / (int)sizeof(S)) == 0;
    const bool async_fill = chunked || sizeof(S) >= 4;

    // seam columns: the box elements a thread copies are the same in every plane;
    // their wrapped x-y slot offsets (-1: off a non-periodic box) are fixed here
    constexpr int NJ = (BOX + NT - 1) / NT;
    int xy_off[NJ];
#pragma unroll
    for (int j = 0; j < NJ; j++) {
        const int e = tid + j * NT;
        int sx = X0 - XA + e % BW, sy = Y0 - 2 + e / BW;
        const bool ok = e < BOX && wrap_coord(sx, g.n[0], g.per[0]) && wrap_coord(sy, g.n[1], g.per[1]);
        xy_off[j] = ok ? sx + g.px * sy : -1;
    }
    __shared__ volatile int s_timeout;  // set by a thread whose stage wait gave up
    if (tid == 0) s_timeout = 0;
    if (tid == NT - 32) {
        tma::mbar_init(&bar[0], 1);
        tma::mbar_init(&bar[1], 1);
        tma::mbar_init(&bar[2], NW);  // the ring's split barrier: one arrival per warp and plane
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    const int K = ze - zb + 2;  // planes zb-1 .. ze: macros of all, collisions of zb .. ze-1
    // class of plane k: a plane off a non-periodic box counts as a hole plane (no stage)
    auto plane_of = [&](int k) { return zb - 1 + k; };
    const PlaneRule rule(Lv, X0, Y0, TX, TY);
    auto class_of = [&](int k) {
        const int p = plane_of(k);
        if (!g.per[2] && (p < 0 || p >= g.n[2])) return (int)LOAD_HOLE;
        return rule(p);
    };
    unsigned phase = 0u, pending = 0u;  // per stage: parity of the next wait, copy in flight
    auto issue = [&](int k, int cls_k) {
        if (cls_k == LOAD_HOLE) return;
        if (k == withhold_k && blin == withhold_block) return;  // test hook: this stage never fills
        const int s = k & 1, p = plane_of(k);
        S *dst = stage(s);
        if (!seam) {
            // the last warp issues the copies, one run of populations per lane, after its
            // lane 0 has armed the stage's barrier with the byte count of all of them
            if (tid >= NT - 32) {
                const int lane = tid & 31;
                if (lane == 0) tma::mbar_expect_tx(&bar[s], (unsigned)G::stage_bytes);
                __syncwarp();
                if (lane < kRuns) {
                    int i0 = 0, mi = 0;
                    static_for<kRuns>([&](auto jc) {
                        constexpr int j = decltype(jc)::value;
                        if (lane == j) {
                            i0 = run_start(j);
                            mi = depth_map(run_len(j));
                        }
                    });
                    const int cz = ((kCzPlus >> i0) & 1u) ? 1 : (((kCzMinus >> i0) & 1u) ? -1 : 0);
                    int zq = p - cz;
                    if (g.per[2]) zq = zq < 0 ? zq + g.n[2] : (zq >= g.n[2] ? zq - g.n[2] : zq);
                    tma::fence_proxy_async();
                    tma::load4d(dst + i0 * BOX, &tmaps.m[mi], &bar[s], X0 - XA, Y0 - 2, zq, i0);
                }
            }
            pending |= 1u << s;
        } else if (chunked) {
            // 16-byte asynchronous copies with wrapped coordinates: a box row is whole
            // 16-byte chunks, and with a periodic x extent of whole chunks a chunk never
            // straddles the seam (completed before the barrier that precedes the use)
            int zo[3];  // slot offset of planes p+1, p, p-1 (c_z = -1, 0, 1); -1 off the box
#pragma unroll
            for (int c = 0; c < 3; c++) {
                int sz = p + 1 - c;
                zo[c] = wrap_coord(sz, g.n[2], g.per[2]) ? n01 * sz : -1;
            }
            constexpr int CE = 16 / (int)sizeof(S), CPR = BW / CE, NCH = CPR * G::BH;
            static_assert(BW % CE == 0 && NCH <= NT, "one chunk per thread and population");
            if (tid < NCH) {
                const int row = tid / CPR, cc = tid % CPR;
                int sx = X0 - XA + cc * CE, sy = Y0 - 2 + row;
                // off a non-periodic x extent: a chunk that starts inside the row ends
                // inside its padded pitch (px is a multiple of 8 nodes)
                const bool okxy = wrap_coord(sy, g.n[1], g.per[1]) &&
                                  (g.per[0] ? wrap_coord(sx, g.n[0], 1) : (sx >= 0 && sx < g.n[0]));
                const int oxy = okxy ? sx + g.px * sy : 0;
                static_for<Q>([&](auto ic) {
                    constexpr int i = decltype(ic)::value;
                    const int z0 = zo[L::c(i, 2) + 1];
                    const bool ok = okxy && z0 >= 0;
                    tma::cp_async<16>(dst + i * BOX + row * BW + cc * CE,
                                      fsrc + (long long)i * g.pitch + (ok ? oxy + z0 : 0), ok);
                });
            }
            tma::cp_async_commit();
        } else {
            // element copies with wrapped coordinates (asynchronous for 4- and 8-byte
            // types; completed before the barrier that precedes the stage's use)
            int zo[3];
#pragma unroll
            for (int c = 0; c < 3; c++) {
                int sz = p + 1 - c;
                zo[c] = wrap_coord(sz, g.n[2], g.per[2]) ? n01 * sz : -1;
            }
            static_for<Q>([&](auto ic) {
                constexpr int i = decltype(ic)::value;
                const S *src = fsrc + (long long)i * g.pitch;
                const int z0 = zo[L::c(i, 2) + 1];
#pragma unroll
                for (int j = 0; j < NJ; j++) {
                    const int e = tid + j * NT;
                    if (e >= BOX) break;
                    const bool ok = xy_off[j] >= 0 && z0 >= 0;
                    if constexpr (sizeof(S) >= 4)
                        tma::cp_async<(int)sizeof(S)>(dst + i * BOX + e, ok ? src + xy_off[j] + z0 : src, ok);
                    else
                        dst[i * BOX + e] = ok ? src[xy_off[j] + z0] : S();
                }
            });
            if constexpr (sizeof(S) >= 4) tma::cp_async_commit();
        }
    };

    // tags of the own and halo node of plane k (general planes only)
    auto tags_of = [&](int k, int &t_own, int &t_halo) {
        const int p = plane_of(k);
        int ox = x, oy = y, oz = p;
        const bool ok = wrap_coord(ox, g.n[0], g.per[0]) && wrap_coord(oy, g.n[1], g.per[1]) &&
                        wrap_coord(oz, g.n[2], g.per[2]);
        t_own = ok ? Lv.tag[box_index(g, ox, oy, oz)] : TAG_HOLE;
        t_halo = TAG_HOLE;
        if (hb >= 0) {
            int qx = X0 + hx - 1, qy = Y0 + hy - 1, qz = p;
            const bool hok = wrap_coord(qx, g.n[0], g.per[0]) && wrap_coord(qy, g.n[1], g.per[1]) &&
                             wrap_coord(qz, g.n[2], g.per[2]);
            t_halo = hok ? Lv.tag[box_index(g, qx, qy, qz)] : TAG_HOLE;
        }
    };

    // moments of a node's populations pulled from stage st at box offset b
    auto stage_moments = [&](const S *st, int b, R (&m)[10], auto only_j) {
        R v[Q];
        static_for<Q>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            v[i] = raw<S>(st[i * BOX + b - L::c(i, 1) * BW - L::c(i, 0)]);
        });
        pair_moments19<R, decltype(only_j)::value>(v, m);
        if constexpr (SHIFT && PLAIN) {
            // the moments of s_i = w_i: 1, 0, c_s^2 I
            m[0] += R(1);
            if constexpr (!decltype(only_j)::value) {
                m[4] += R(1.0 / 3.0);
                m[5] += R(1.0 / 3.0);
                m[6] += R(1.0 / 3.0);
            }
        } else if constexpr (SHIFT) {
            constexpr int nm = decltype(only_j)::value ? 4 : 10;
#pragma unroll
            for (int q = 0; q < nm; q++) m[q] += R(Lv.smom[q]);
        }
    };
    const R *tpop = (const R *)Lv.if_pop, *tmac = (const R *)Lv.if_mac;

    // state carried from plane to plane: the node of plane p - 1 (tag, rho, Pq = Pi - cs2
    // sum f I); z values of planes p - 2 and p - 1
    int tc = TAG_HOLE;
    R rho_c = R(1), pq_c[6] = {0, 0, 0, 0, 0, 0};
    R zm[9], z0[9];
#pragma unroll
    for (int q = 0; q < 9; q++) zm[q] = z0[q] = R(0);

    int nt_own = TAG_HOLE, nt_halo = TAG_HOLE;  // tags of the next general plane (loaded one plane ahead)
    int c0 = class_of(0), c1 = class_of(1);     // classes of planes k, k + 1 (K >= 3)
    issue(0, c0);
    issue(1, c1);
    if (seam) {  // stages filled by copies from the threads
        if (async_fill) tma::cp_async_wait_all();
        __syncthreads();
    }
    if (c0 == LOAD_GENERAL) tags_of(0, nt_own, nt_halo);
    for (int k = 0; k < K; k++) {
        const int p = plane_of(k);
        const int s = k & 1;
        const int cls = c0;
        const int t_own = cls == LOAD_FAST ? TAG_BULK : nt_own, t_halo = cls == LOAD_FAST ? TAG_BULK : nt_halo;
        if (k + 1 < K && c1 == LOAD_GENERAL) tags_of(k + 1, nt_own, nt_halo);
        bool ok = true;
        if (cls != LOAD_HOLE && !seam) {
            ok = tma::mbar_wait(&bar[s], (phase >> s) & 1u, limit_ns);
            phase ^= 1u << s;
            if (ok) pending &= ~(1u << s);
        }
        R *rs = ring + (size_t)(p & 1) * HP * NV;  // ring slot of plane p
        // own node of plane p: moments (kept for its collision one plane later), u and Psi
        int tn = TAG_HOLE;
        const R cs2 = R(1) / R(3);
        R rho_n = R(1), pq_n[6] = {0, 0, 0, 0, 0, 0}, un[3] = {0, 0, 0};
        if (cls != LOAD_HOLE && ok) {
            tn = t_own;
            if (tn == TAG_BULK) {
                R m[10];
                stage_moments(stage(s), own_b, m, std::false_type{});
                rho_n = m[0];
                const R inv = recip(m[0]);
#pragma unroll
                for (int a = 0; a < 3; a++) un[a] = m[1 + a] * inv;
#pragma unroll
                for (int q = 0; q < 6; q++) pq_n[q] = q < 3 ? m[4 + q] - cs2 * m[0] : m[4 + q];
            } else if (tn >= 0) {
                R f[Q];
#pragma unroll
                for (int i = 0; i < Q; i++) f[i] = tpop[(long long)i * Lv.nif + tn];
                R m[10];
                pair_moments19<R>(f, m);
#pragma unroll
                for (int q = 0; q < 6; q++) pq_n[q] = q < 3 ? m[4 + q] - cs2 * m[0] : m[4 + q];
                rho_n = tmac[tn];
#pragma unroll
                for (int a = 0; a < 3; a++) un[a] = tmac[(long long)(1 + a) * Lv.nif + tn];
            }
        }
        R zp[9];
        {
            R rv[12];
            psi_ring<R>(rho_n, un, rv, zp);
            ring_store<R>(rs + hs * NV, rv);
        }
        if (hb >= 0) {
            R hr = R(1), hu[3] = {R(0), R(0), R(0)};
            if (cls != LOAD_HOLE && ok) {
                if (t_halo == TAG_BULK) {
                    R m[10];
                    stage_moments(stage(s), halo_b, m, std::true_type{});
                    const R ir = recip(m[0]);
                    hr = m[0];
                    hu[0] = m[1] * ir;
                    hu[1] = m[2] * ir;
                    hu[2] = m[3] * ir;
                } else if (t_halo >= 0) {
                    hr = tmac[t_halo];
#pragma unroll
                    for (int a = 0; a < 3; a++) hu[a] = tmac[(long long)(1 + a) * Lv.nif + t_halo];
                }
            }
            R rv[12], zv[9];
            psi_ring<R>(hr, hu, rv, zv);
            ring_store<R>(rs + hb * NV, rv);
        }
        if (!in_xy) tn = TAG_HOLE;  // a position past a periodic seam only feeds the halo
        if (seam && async_fill) tma::cp_async_wait_all();  // the copies of the next stage, issued one plane ago
        if (!ok) s_timeout = 1;
        // in-plane differences of the node of plane p - 1 from the ring slot of plane
        // p - 1 (complete since the previous wait; nobody overwrites it before this warp
        // arrives below)
        R sc[11];  // S_xx, S_yy, S_xy, d_x u_z, d_y u_z, C_0..C_5 (x and y parts)
        if (k >= 2 && tc == TAG_BULK) {
            const R *rq = ring + (size_t)((p - 1) & 1) * HP * NV;
            R xp[12], xm[12], yp[12], ym[12];
            ring_load<R>(rq + (hs + 1) * NV, xp);
            ring_load<R>(rq + (hs - 1) * NV, xm);
            ring_load<R>(rq + (hs + HX) * NV, yp);
            ring_load<R>(rq + (hs - HX) * NV, ym);
            auto dx = [&](int q) { return (xp[q] - xm[q]) * R(0.5); };
            auto dy = [&](int q) { return (yp[q] - ym[q]) * R(0.5); };
            sc[0] = dx(0);
            sc[1] = dy(1);
            sc[2] = R(0.5) * (dy(0) + dx(1));
            sc[3] = dx(2);
            sc[4] = dy(2);
            sc[5] = dx(RV_PXXX) + dy(RV_PXXY);
            sc[6] = dx(RV_PXYY) + dy(RV_PYYY);
            sc[7] = dx(RV_PXZZ) + dy(RV_PYZZ);
            sc[8] = dx(RV_PXXY) + dy(RV_PXYY);
            sc[9] = dx(RV_PXXZ) + dy(RV_PXYZ);
            sc[10] = dx(RV_PXYZ) + dy(RV_PYYZ);
        }
        // split barrier (mbarrier 2, phase k): the warp's ring values of plane p are
        // published by its arrival; the collision of plane p - 1 below reads nothing
        // another thread writes in this iteration, so it runs before the wait
        __syncwarp();
        if ((tid & 31) == 0) mbar_arrive(&bar[2]);

        // collide plane p - 1: z differences from the z values of planes p and p - 2
        if (k >= 2 && tc != TAG_HOLE) {
            const int z = p - 1;
            R Sv[6], Cv[6];
            if (tc == TAG_BULK) {
                R dz[9];
#pragma unroll
                for (int q = 0; q < 9; q++) dz[q] = (zp[q] - zm[q]) * R(0.5);
                Sv[0] = sc[0];
                Sv[1] = sc[1];
                Sv[2] = dz[2];
                Sv[3] = sc[2];
                Sv[4] = R(0.5) * (dz[0] + sc[3]);
                Sv[5] = R(0.5) * (dz[1] + sc[4]);
                Cv[0] = sc[5] + dz[ZV_PXXZ];
                Cv[1] = sc[6] + dz[ZV_PYYZ];
                Cv[2] = sc[7] + dz[ZV_PZZZ];
                Cv[3] = sc[8] + dz[ZV_PXYZ];
                Cv[4] = sc[9] + dz[ZV_PXZZ];
                Cv[5] = sc[10] + dz[ZV_PYZZ];
            } else {
                // interface node: S and C from its table row (TF rows by the gradient
                // launch, hanging-node rows interpolated from them by k_ie_sc)
                const R *tS = (const R *)Lv.if_S, *tC = (const R *)Lv.if_C;
#pragma unroll
                for (int q = 0; q < 6; q++) {
                    Sv[q] = tS[(long long)q * Lv.nif + tc];
                    Cv[q] = tC[(long long)q * Lv.nif + tc];
                }
            }
            S *dst = fdst + (x + g.px * y + (long long)n01 * z);
            hrr_pairs19<R, SHIFT, PLAIN>(rho_c, z0, pq_c, Sv, Cv, tau, om, sigma, spsi, Lv.she, Lv.sho,
                                  [&](auto ic, R v) {
                                      constexpr int i = decltype(ic)::value;
                                      if constexpr (SHIFT) dst[(long long)i * pitch] = __float2half_rn(v);
                                      else dst[(long long)i * pitch] = v;
                                  });
        }
        if (!tma::mbar_wait(&bar[2], (unsigned)k & 1u, limit_ns)) s_timeout = 1;  // a warp that never arrives
        if (s_timeout) {
            // a copy did not arrive in time: report, drain what is in flight, stop
            if (tid == 0) atomicOr(status, ST_TIMEOUT);
            for (int q = 0; q < 2; q++)
                if ((pending >> q) & 1u) tma::mbar_wait(&bar[q], (phase >> q) & 1u, limit_ns);
            return;
        }
        const int c2 = k + 2 < K ? class_of(k + 2) : (int)LOAD_HOLE;
        if (k + 2 < K) issue(k + 2, c2);  // into the stage every thread has read
        c0 = c1;
        c1 = c2;

        tc = tn;
        rho_c = rho_n;
#pragma unroll
        for (int q = 0; q < 6; q++) pq_c[q] = pq_n[q];
#pragma unroll
        for (int q = 0; q < 9; q++) {
            zm[q] = z0[q];
            z0[q] = zp[q];
        }
    }
}

}  // namespace lbmg
