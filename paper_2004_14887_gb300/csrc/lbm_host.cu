// Host side of the GB300 direct-coupling multi-level lattice Boltzmann library:
// hierarchy geometry, node classification (Sec. 3.2 sets, App. B corners), interface
// tables, the recursive 2:1 sub-cycling schedule of Sec. 3.5 issued as kernel
// launches (captured once per coarse-step phase into CUDA graphs), and the C-ABI
// declared in include/lbm.h.
#include <cuda.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>  // header-only; the markers cost nothing without a profiler

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_kernels.cuh"
#include "lbm_bulk3d.cuh"

using namespace lbmg;

namespace {

thread_local std::string g_create_error;

// NVTX range for profiler timelines (lbm_advance, coarse steps, level sub-steps)
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};
const char *const kLevelRange[LBM_MAX_LEVELS] = {"level 0 step", "level 1 step", "level 2 step", "level 3 step"};

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

struct Level {
    int64_t n[3] = {1, 1, 1}, off[3] = {0, 0, 0};
    int per[3] = {1, 1, 1};
    long long N = 0, pitch = 0;  // dense node count; elements between population planes
    long long px = 1, NS = 0;     // row pitch (x extent padded to 8 nodes) and box slots px*ny*nz
    double tau = 0.5;
    std::vector<uint8_t> cls;
    std::vector<int> tag;
    std::vector<unsigned char> tile_flag;
    // per-tile classes of the 2-D bulk kernel for each tile shape, node by node: levels
    // a staircase region touches (the geometric tile rule assumes boxes)
    bool use_tflag = false;
    std::vector<unsigned char> tflag[LBM_TILE_CONFIGS];
    unsigned char *d_tflag[LBM_TILE_CONFIGS] = {};
    int tiles[3] = {1, 1, 1};
    int nTFP = 0, nIE = 0, nTFC = 0, nif = 0;
    int tile_cfg = 0;  // D2Q9 bulk tile shape (kTileCfgs), chosen by lbm_autotune
    int zc = 1;        // D3Q19: planes per z chunk of the bulk kernel
    TMaps tmap[2];  // D3Q19: bulk tensor copy maps of f[0], f[1] (boxes of 1, 2, 4, 5 populations)
    int64_t n_active = 0;
    // child-box in this level's node coordinates, for volume weights
    bool has_child = false;
    int64_t child_lo[3] = {0, 0, 0}, child_hi[3] = {0, 0, 0};
    int child_per[3] = {1, 1, 1};
    // device
    void *f[2] = {nullptr, nullptr};
    int *d_tag = nullptr;
    void *if_pop = nullptr, *if_mac = nullptr, *if_S = nullptr, *if_C = nullptr;
    double *d_wnode = nullptr;
};

struct Iface {  // between coarse level l-1 and fine level l
    std::vector<long long> tf_fine, tf_coarse, ie_fine, ring_coarse;
    std::vector<int> tf_ridx;
    std::vector<unsigned int> tf_kf, tf_kc, tf_gc, ie_kf;
    std::vector<signed char> tf_rkind;
    std::vector<int> ie_nst, ie_st;
    std::vector<double> ie_w;
    IfaceDev dev{};
    double R = 0.5;
};

}  // namespace

struct lbm_hierarchy {
    lbm_hierarchy_desc d{};
    int Q = 9, D = 2, nl = 1;
    Level lev[LBM_MAX_LEVELS];
    Iface ifc[LBM_MAX_LEVELS];  // ifc[l] couples level l-1 and level l (l >= 1)
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = 0;  // the CUDA device current at creation; the handle's arrays live there
    // second stream: a level's TF-gradient / hanging-node launch runs beside its child
    // level's sub-steps (fork and join events per level; captured as graph branches)
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork[LBM_MAX_LEVELS] = {}, ev_join[LBM_MAX_LEVELS] = {};
    // one more stream per level with a child: the level's bulk launch starts once its
    // child's sync sub-step has written this level's child-TF rows (ev_parent) and runs
    // beside the child's rest; a stream per level lets a coarse level's bulk launch run
    // beside its grandchild's sub-steps instead of queueing behind its child's bulk launch
    cudaStream_t side2[LBM_MAX_LEVELS] = {};
    cudaEvent_t ev_parent[LBM_MAX_LEVELS] = {}, ev_bulk[LBM_MAX_LEVELS] = {};
    std::vector<DevBuf> bufs;
    int64_t device_bytes = 0;
    int *d_status = nullptr, *d_maxit = nullptr;
    int if_mode = LBM_IFACE_AUTO;  // interface thread mapping (lbm_set_interface_mapping)
    // staircase regions (lbm_create_hierarchy_masked): per level, the refined parent
    // cells of its box (x fastest; empty: the whole box)
    std::vector<uint8_t> mask[LBM_MAX_LEVELS];
    bool masked = false;
    // test hook of the 3-D bulk kernel's bounded waits (lbm_debug_withhold_copy)
    int withhold_level = -1, withhold_block = -1, withhold_k = -1;
    unsigned long long withhold_limit_ns = 0;
    float shift[19] = {};          // FP16-shifted storage: f_i - shift[i] (f_i^eq(1, u_shift))
    bool plain_shift = false;      // FP16 storage with u_shift = 0 (shift[i] = w_i)
    double *d_partial = nullptr, *d_red = nullptr;
    int red_blocks = 0;
    long long ncoarse = 0;  // coarse steps done since init
    std::map<int, cudaGraphExec_t> graphs;
    std::map<int, int64_t> graph_launches;
    int64_t launches = 0;
    int64_t launch_counter = 0;  // launches issued by the current issue pass
    bool timing = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<int, int>> ev_pairs;  // (level, event index of the start)
    double timing_ms[LBM_MAX_LEVELS] = {0, 0, 0, 0};
    int64_t timing_launches[LBM_MAX_LEVELS] = {0, 0, 0, 0};
    std::string err;
    // probes
    ProbeDev probes{};
    LevelDev *d_levs = nullptr;     // level views for the probe kernel
    long long *d_kstep = nullptr;   // per-level step index of the current state
    int64_t probe_rows = 0;
    // batched hierarchies (lbm_create_batch): the batch owns its members
    std::vector<lbm_hierarchy *> members;
    lbm_hierarchy *batch = nullptr;  // set on members
    BatchDev bdev{};
    BatchPhase *d_phases = nullptr;
    std::vector<BatchPhase> phases;                    // the same on the host
    std::vector<int> work_bulk, work_rh, work_gi;      // per level: work items of a phase (all members)
    int batch_path = LBM_BATCH_PERSISTENT;             // launch structure of lbm_advance on a batch
    int nphases = 0;
    int batch_grid = 0;
};

namespace {

int fail(lbm_h h, int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (h) h->err = buf;
    else g_create_error = buf;
    return code;
}

#define CK(call)                                                                                  \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess) return fail(h, LBM_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

void *dev_alloc(lbm_h h, size_t bytes)
{
    bytes = (bytes + 255) & ~(size_t)255;
    if (bytes == 0) bytes = 256;
    void *p = nullptr;
    if (h->d.alloc) p = h->d.alloc(bytes, h->d.alloc_ctx);
    else if (cudaMalloc(&p, bytes) != cudaSuccess) p = nullptr;
    if (p) {
        h->bufs.push_back({p, bytes});
        h->device_bytes += (int64_t)bytes;
    }
    return p;
}

// short-lived staging buffers go through the same allocator as the handle's arrays
void *tmp_alloc(lbm_h h, size_t bytes)
{
    void *p = nullptr;
    if (h->d.alloc) p = h->d.alloc(bytes, h->d.alloc_ctx);
    else if (cudaMalloc(&p, bytes) != cudaSuccess) p = nullptr;
    return p;
}
void tmp_free(lbm_h h, void *p)
{
    if (!p) return;
    if (h->d.free) h->d.free(p, h->d.alloc_ctx);
    else cudaFree(p);
}

template <typename T>
T *upload(lbm_h h, const std::vector<T> &v, bool *ok)
{
    T *p = (T *)dev_alloc(h, std::max<size_t>(1, v.size()) * sizeof(T));
    if (!p) {
        *ok = false;
        return nullptr;
    }
    if (!v.empty() && cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess)
        *ok = false;
    return p;
}

int64_t emod(int64_t a, int64_t n)
{
    int64_t r = a % n;
    return r < 0 ? r + n : r;
}

int lat_c(int Q, int i, int a) { return Q == 9 ? Lat<9>::c(i, a) : Lat<19>::c(i, a); }

size_t store_size(int storage) { return storage == LBM_F64 ? 8 : (storage == LBM_F32 ? 4 : 2); }
// arithmetic type of the storage: FP64 for FP64 storage, FP32 otherwise
size_t arith_size(int storage) { return storage == LBM_F64 ? 8 : 4; }

// box coordinates of linear indices, [n][3] int32
std::vector<int> coords3(const Level &v, const std::vector<long long> &idx)
{
    std::vector<int> out(idx.size() * 3);
    for (size_t k = 0; k < idx.size(); k++) {
        out[3 * k] = (int)(idx[k] % v.n[0]);
        out[3 * k + 1] = (int)((idx[k] / v.n[0]) % v.n[1]);
        out[3 * k + 2] = (int)(idx[k] / (v.n[0] * v.n[1]));
    }
    return out;
}

// linear index of global level-l coordinates p, or -1 if not a node of level l
long long node_of(const lbm_h h, int l, const int64_t *p)
{
    const Level &v = h->lev[l];
    int64_t q[3];
    for (int a = 0; a < 3; a++) {
        q[a] = p[a] - v.off[a];
        if (v.per[a]) q[a] = emod(q[a], v.n[a]);
        else if (q[a] < 0 || q[a] >= v.n[a]) return -1;
    }
    long long idx = q[0] + v.n[0] * (q[1] + v.n[1] * q[2]);
    if (v.cls[idx] == LBM_NODE_HOLE) return -1;
    return idx;
}

void global_of(const Level &v, long long idx, int64_t *p)
{
    p[0] = idx % v.n[0] + v.off[0];
    p[1] = (idx / v.n[0]) % v.n[1] + v.off[1];
    p[2] = idx / (v.n[0] * v.n[1]) + v.off[2];
}

// ------------------------------------------------------------------ geometry
// Does level l (>= 1) refine the cell of its parent level l-1 with lower corner c
// (global level-(l-1) coordinates)?  The box's cells on every axis it does not span,
// any cell on an axis it spans, and of those the ones its mask marks.
bool refines(const lbm_h h, int l, const int64_t *c)
{
    const lbm_hierarchy_desc &d = h->d;
    const Level &pv = h->lev[l - 1];
    int64_t q[3] = {0, 0, 0}, ext[3] = {1, 1, 1};
    for (int a = 0; a < h->D; a++) {
        int64_t ca = c[a];
        if (pv.per[a]) ca = pv.off[a] + emod(ca - pv.off[a], pv.n[a]);
        if (h->lev[l].per[a]) continue;
        const int64_t psc = (int64_t)1 << (l - 1), lo = d.box_lo[l][a] * psc, hi = d.box_hi[l][a] * psc;
        if (ca < lo || ca >= hi) return false;
        q[a] = ca - lo;
        ext[a] = hi - lo;
    }
    if (h->mask[l].empty()) return true;
    return h->mask[l][(size_t)(q[0] + ext[0] * (q[1] + ext[1] * q[2]))] != 0;
}

// refined cells (by level l) among the 2^D cells around node p of level l-1; *tot = 2^D
int refined_around(const lbm_h h, int l, const int64_t *p, int *tot)
{
    int cnt = 0;
    *tot = 1 << h->D;
    for (int k = 0; k < *tot; k++) {
        int64_t c[3] = {p[0], p[1], p[2]};
        for (int a = 0; a < h->D; a++) c[a] -= (k >> a) & 1;
        cnt += refines(h, l, c);
    }
    return cnt;
}

// refined cells among the parent cells that node p of level l touches (two per even
// coordinate, one per odd one); *tot = their number
int refined_touched(const lbm_h h, int l, const int64_t *p, int *tot)
{
    int64_t lo[3] = {0, 0, 0}, cnt_a[3] = {1, 1, 1};
    for (int a = 0; a < h->D; a++) {
        if (emod(p[a], 2) == 0) {
            lo[a] = p[a] / 2 - 1;
            cnt_a[a] = 2;
        } else {
            lo[a] = (p[a] - 1) / 2;
        }
    }
    int cnt = 0;
    *tot = 0;
    for (int64_t k2 = 0; k2 < cnt_a[2]; k2++)
        for (int64_t k1 = 0; k1 < cnt_a[1]; k1++)
            for (int64_t k0 = 0; k0 < cnt_a[0]; k0++) {
                const int64_t c[3] = {lo[0] + k0, lo[1] + k1, lo[2] + k2};
                cnt += refines(h, l, c);
                (*tot)++;
            }
    return cnt;
}

int build_geometry(lbm_h h)
{
    const lbm_hierarchy_desc &d = h->d;
    for (int l = 0; l < h->nl; l++) {
        Level &v = h->lev[l];
        for (int a = 0; a < 3; a++) {
            if (a >= h->D) {
                v.n[a] = 1;
                v.off[a] = 0;
                v.per[a] = 1;
                continue;
            }
            if (l == 0) {
                v.n[a] = d.coarse_n[a];
                v.off[a] = 0;
                v.per[a] = 1;
                continue;
            }
            const int64_t lo = d.box_lo[l][a], hi = d.box_hi[l][a];
            if (lo == 0 && hi == d.coarse_n[a]) {
                if (!h->lev[l - 1].per[a]) return fail(nullptr, LBM_ERR_BAD_DESC, "level %d spans axis %d but its parent does not", l, a);
                v.n[a] = d.coarse_n[a] << l;
                v.off[a] = 0;
                v.per[a] = 1;
                continue;
            }
            const int64_t psc = (int64_t)1 << (l - 1);
            if (hi <= lo) return fail(nullptr, LBM_ERR_BAD_DESC, "level %d: empty patch on axis %d", l, a);
            if ((hi - lo) * psc < 4) return fail(nullptr, LBM_ERR_BAD_DESC, "level %d: a face needs >= 4 parent cells", l);
            if (h->lev[l - 1].per[a]) {
                if (lo * psc < 4 || (d.coarse_n[a] - hi) * psc < 4)
                    return fail(nullptr, LBM_ERR_BAD_DESC, "level %d: patch within 4 parent cells of the periodic seam", l);
            } else {
                const int64_t plo = d.box_lo[l - 1][a], phi = d.box_hi[l - 1][a];
                if ((lo - plo) * psc < 4 || (phi - hi) * psc < 4)
                    return fail(nullptr, LBM_ERR_BAD_DESC, "level %d: patch needs 4 parent cells of margin", l);
            }
            v.n[a] = ((hi - lo) << l) + 1;
            v.off[a] = lo << l;
            v.per[a] = 0;
        }
        if (l > 0) {
            bool all_span = true;
            for (int a = 0; a < h->D; a++) all_span = all_span && v.per[a];
            if (all_span) return fail(nullptr, LBM_ERR_BAD_DESC, "level %d spans every axis: refine level 0 instead", l);
        }
        v.N = (long long)v.n[0] * v.n[1] * v.n[2];
        // rows padded to 8 nodes: every row starts 16-byte aligned in each storage type
        // (bulk tensor copies need 16-byte strides); padding slots are holes
        v.px = (v.n[0] + 7) / 8 * 8;
        v.NS = v.px * v.n[1] * v.n[2];
        v.pitch = (v.NS + 31) / 32 * 32;
        v.tau = l == 0 ? 0.5 + 3.0 * d.nu0 : 2.0 * h->lev[l - 1].tau - 0.5;
        if (l + 1 < h->nl) {
            v.has_child = true;
            for (int a = 0; a < 3; a++) {
                const int64_t lo = d.box_lo[l + 1][a], hi = d.box_hi[l + 1][a];
                v.child_per[a] = (a >= h->D) || (lo == 0 && hi == d.coarse_n[a]);
                v.child_lo[a] = lo << l;
                v.child_hi[a] = hi << l;
            }
        }
    }
    // staircase regions: 2-D, the finest level only, a box that spans no axis, and no
    // two refined cells that meet at a corner only
    for (int l = 1; l < h->nl; l++) {
        if (h->mask[l].empty()) continue;
        if (h->D != 2) return fail(nullptr, LBM_ERR_BAD_DESC, "refinement masks are 2-D only");
        if (l + 1 < h->nl) return fail(nullptr, LBM_ERR_BAD_DESC, "a refinement mask is allowed on the finest level only");
        for (int a = 0; a < h->D; a++)
            if (h->lev[l].per[a]) return fail(nullptr, LBM_ERR_BAD_DESC, "a masked level spans no axis");
        const int64_t psc = (int64_t)1 << (l - 1);
        for (int64_t cy = d.box_lo[l][1] * psc; cy <= d.box_hi[l][1] * psc; cy++)
            for (int64_t cx = d.box_lo[l][0] * psc; cx <= d.box_hi[l][0] * psc; cx++) {
                const int64_t c00[3] = {cx - 1, cy - 1, 0}, c10[3] = {cx, cy - 1, 0}, c01[3] = {cx - 1, cy, 0},
                              c11[3] = {cx, cy, 0};
                const bool a00 = refines(h, l, c00), a10 = refines(h, l, c10), a01 = refines(h, l, c01),
                           a11 = refines(h, l, c11);
                if (a00 == a11 && a10 == a01 && a00 != a10)
                    return fail(nullptr, LBM_ERR_BAD_DESC, "two refined cells meet at a corner only");
            }
    }
    // classes (Sec. 3.2; App. B at staircase corners) from the refined cells around a
    // node: a node whose cells the next level all refines is a hole, one with some
    // refined cells is co-located with a TF node of the child; a node of a refined level
    // that touches a cell its level does not refine lies on the interface (TF when
    // co-located with a parent node, else hanging); one touching no refined cell is not
    // a node of the level (a hole of the box)
    for (int l = 0; l < h->nl; l++) {
        Level &v = h->lev[l];
        v.cls.assign(v.N, LBM_NODE_BULK);
        for (long long idx = 0; idx < v.N; idx++) {
            int64_t p[3];
            global_of(v, idx, p);
            uint8_t c = LBM_NODE_BULK;
            if (l + 1 < h->nl) {
                int tot = 0;
                const int cnt = refined_around(h, l + 1, p, &tot);
                if (cnt == tot) c = LBM_NODE_HOLE;
                else if (cnt > 0) c = LBM_NODE_TF_CHILD;
            }
            if (l > 0) {
                int tot = 0;
                const int cnt = refined_touched(h, l, p, &tot);
                bool even = true;
                for (int a = 0; a < h->D; a++)
                    if (emod(p[a], 2) != 0) even = false;
                if (cnt == 0) c = LBM_NODE_HOLE;
                else if (cnt < tot && c == LBM_NODE_BULK) c = even ? LBM_NODE_TF_PARENT : LBM_NODE_HANGING;
                else if (cnt < tot) return fail(nullptr, LBM_ERR_BAD_DESC, "level %d's interface meets its child's region", l);
            }
            v.cls[idx] = c;
        }
        v.n_active = 0;
        for (long long idx = 0; idx < v.N; idx++) v.n_active += v.cls[idx] != LBM_NODE_HOLE;
    }
    return LBM_OK;
}

unsigned int full_mask(int Q) { return (Q >= 32) ? 0xffffffffu : ((1u << Q) - 1u); }

// fine-known / coarse-known masks of a node: population i is known on a level if the
// node x - c_i (x/2 - c_i on the parent) exists there (Sec. 3.2 sets, App. B)
unsigned int known_mask(const lbm_h h, int l, const int64_t *p)
{
    unsigned int m = 0;
    for (int i = 0; i < h->Q; i++) {
        int64_t s[3] = {p[0] - lat_c(h->Q, i, 0), p[1] - lat_c(h->Q, i, 1), p[2] - lat_c(h->Q, i, 2)};
        if (node_of(h, l, s) >= 0) m |= 1u << i;
    }
    return m;
}

int build_interfaces(lbm_h h)
{
    const int Q = h->Q, D = h->D;
    const unsigned int all = full_mask(Q);
    for (int l = 1; l < h->nl; l++) {
        Level &F = h->lev[l];
        Level &C = h->lev[l - 1];
        Iface &I = h->ifc[l];
        I.R = 0.5 * F.tau / C.tau;
        std::vector<int> tf_of(F.N, -1);
        // TF and hanging nodes of the fine level in index order
        for (long long idx = 0; idx < F.N; idx++) {
            int64_t p[3];
            global_of(F, idx, p);
            if (F.cls[idx] == LBM_NODE_TF_PARENT) {
                int64_t pc[3] = {p[0] / 2, p[1] / 2, p[2] / 2};
                const long long cidx = node_of(h, l - 1, pc);
                if (cidx < 0 || C.cls[cidx] != LBM_NODE_TF_CHILD)
                    return fail(nullptr, LBM_ERR_BAD_DESC, "TF node without a co-located coarse node");
                const unsigned int kf = known_mask(h, l, p), kc = known_mask(h, l - 1, pc);
                if ((kf | kc) != all) return fail(nullptr, LBM_ERR_BAD_DESC, "TF node misses a population on both levels");
                tf_of[idx] = (int)I.tf_fine.size();
                I.tf_fine.push_back(idx);
                I.tf_coarse.push_back(cidx);
                I.tf_kf.push_back(kf);
                I.tf_kc.push_back(kc);
                // Table 1: DC2 takes coarse data on P and M^f (= every coarse-known
                // population here), DC1 on M^f only
                I.tf_gc.push_back(h->d.dc_variant == 1 ? (all & ~kf) : kc);
            }
        }
        for (long long idx = 0; idx < F.N; idx++)
            if (F.cls[idx] == LBM_NODE_HANGING) {
                int64_t p[3];
                global_of(F, idx, p);
                I.ie_fine.push_back(idx);
                I.ie_kf.push_back(known_mask(h, l, p));
            }
        const int nTF = (int)I.tf_fine.size(), nIE = (int)I.ie_fine.size();
        // gradient stencil references
        std::map<long long, int> ring_of;
        I.tf_rkind.assign((size_t)nTF * 2 * D, RK_FINE);
        I.tf_ridx.assign((size_t)nTF * 2 * D, 0);
        for (int t = 0; t < nTF; t++) {
            int64_t p[3];
            global_of(F, I.tf_fine[t], p);
            for (int b = 0; b < D; b++)
                for (int s = 0; s < 2; s++) {
                    int64_t y[3] = {p[0], p[1], p[2]};
                    y[b] += s == 0 ? 2 : -2;
                    const size_t k = (size_t)t * 2 * D + 2 * b + s;
                    const long long j = node_of(h, l, y);
                    if (j >= 0) {
                        if (F.cls[j] == LBM_NODE_TF_PARENT) {
                            I.tf_rkind[k] = RK_TF;
                            I.tf_ridx[k] = tf_of[j];
                        } else if (F.cls[j] == LBM_NODE_BULK) {
                            I.tf_rkind[k] = RK_FINE;
                            I.tf_ridx[k] = (int)j;
                        } else {
                            return fail(nullptr, LBM_ERR_BAD_DESC, "TF gradient stencil meets a non-bulk fine node");
                        }
                    } else {
                        int64_t yc[3] = {y[0] / 2, y[1] / 2, y[2] / 2};
                        const long long jc = node_of(h, l - 1, yc);
                        if (jc < 0 || C.cls[jc] != LBM_NODE_BULK)
                            return fail(nullptr, LBM_ERR_BAD_DESC, "TF gradient stencil leaves the coarse bulk");
                        auto it = ring_of.find(jc);
                        int r;
                        if (it == ring_of.end()) {
                            r = (int)I.ring_coarse.size();
                            ring_of[jc] = r;
                            I.ring_coarse.push_back(jc);
                        } else {
                            r = it->second;
                        }
                        I.tf_rkind[k] = RK_RING;
                        I.tf_ridx[k] = r;
                    }
                }
        }
        // hanging-node stencils: per odd axis a 4-point 1-D Lagrange set at the
        // mid-point (centred -1/16, 9/16, 9/16, -1/16; one-sided 5/16, 15/16, -5/16, 1/16
        // next to a corner), tensor product over the odd axes
        I.ie_nst.assign(nIE, 0);
        I.ie_st.assign((size_t)nIE * 16, 0);
        I.ie_w.assign((size_t)nIE * 16, 0.0);
        const double wc[4] = {-1.0 / 16, 9.0 / 16, 9.0 / 16, -1.0 / 16};
        const double wo[4] = {5.0 / 16, 15.0 / 16, -5.0 / 16, 1.0 / 16};
        for (int e = 0; e < nIE; e++) {
            int64_t p[3];
            global_of(F, I.ie_fine[e], p);
            int64_t pos[3][4];
            double wt[3][4];
            int cnt[3];
            for (int a = 0; a < 3; a++) {
                if (a >= D || emod(p[a], 2) == 0) {
                    cnt[a] = 1;
                    pos[a][0] = p[a];
                    wt[a][0] = 1.0;
                    continue;
                }
                cnt[a] = 4;
                const int64_t q = p[a] - F.off[a];
                static const int oc[4] = {-3, -1, 1, 3}, olo[4] = {-1, 1, 3, 5}, ohi[4] = {1, -1, -3, -5};
                const int *o = oc;
                const double *w = wc;
                if (D == 2) {
                    // 2-D, boxes and staircases (reading R15): the first of the centred and
                    // the two one-sided 4-point sets along the odd axis made of TF nodes only;
                    // else the 2-point linear set of the TF nodes that end the node's edge
                    const int *cand[3] = {oc, olo, ohi};
                    int pick = -1;
                    for (int k = 0; k < 3 && pick < 0; k++) {
                        bool all_tf = true;
                        for (int m = 0; m < 4 && all_tf; m++) {
                            int64_t y[3] = {p[0], p[1], p[2]};
                            y[a] += cand[k][m];
                            const long long j = node_of(h, l, y);
                            all_tf = j >= 0 && F.cls[j] == LBM_NODE_TF_PARENT;
                        }
                        if (all_tf) pick = k;
                    }
                    if (pick < 0) {
                        cnt[a] = 2;
                        pos[a][0] = p[a] - 1;
                        pos[a][1] = p[a] + 1;
                        wt[a][0] = wt[a][1] = 0.5;
                    } else {
                        for (int k = 0; k < 4; k++) {
                            pos[a][k] = p[a] + cand[pick][k];
                            wt[a][k] = pick == 0 ? wc[k] : wo[k];
                        }
                    }
                    continue;
                }
                if (!F.per[a] && q - 3 < 0) {
                    o = olo;
                    w = wo;
                } else if (!F.per[a] && q + 3 > F.n[a] - 1) {
                    o = ohi;
                    w = wo;
                }
                for (int k = 0; k < 4; k++) {
                    pos[a][k] = p[a] + o[k];
                    wt[a][k] = w[k];
                }
            }
            int m = 0;
            for (int i0 = 0; i0 < cnt[0]; i0++)
                for (int i1 = 0; i1 < cnt[1]; i1++)
                    for (int i2 = 0; i2 < cnt[2]; i2++) {
                        int64_t y[3] = {pos[0][i0], pos[1][i1], pos[2][i2]};
                        const long long j = node_of(h, l, y);
                        if (j < 0 || F.cls[j] != LBM_NODE_TF_PARENT || m >= 16)
                            return fail(nullptr, LBM_ERR_BAD_DESC, "hanging-node stencil does not land on TF nodes");
                        I.ie_st[(size_t)e * 16 + m] = tf_of[j];
                        I.ie_w[(size_t)e * 16 + m] = wt[0][i0] * wt[1][i1] * wt[2][i2];
                        m++;
                    }
            // the kernels read a fixed number of stencil slots: 4 in 2-D, 16 in 3-D
            if (m > (h->D == 2 ? 4 : 16))
                return fail(nullptr, LBM_ERR_BAD_DESC, "internal: a hanging-node stencil of %d points", m);
            I.ie_nst[e] = m;
        }
        F.nTFP = nTF;
        F.nIE = nIE;
        C.nTFC = nTF;
    }
    // tables and tags: [TF_PARENT | HANGING | TF_CHILD]
    for (int l = 0; l < h->nl; l++) {
        Level &v = h->lev[l];
        v.nif = v.nTFP + v.nIE + v.nTFC;
        v.tag.assign(v.N, TAG_BULK);
        for (long long idx = 0; idx < v.N; idx++)
            if (v.cls[idx] == LBM_NODE_HOLE) v.tag[idx] = TAG_HOLE;
        if (l > 0) {
            const Iface &I = h->ifc[l];
            for (int t = 0; t < v.nTFP; t++) v.tag[I.tf_fine[t]] = t;
            for (int e = 0; e < v.nIE; e++) v.tag[I.ie_fine[e]] = v.nTFP + e;
        }
        if (l + 1 < h->nl) {
            const Iface &I = h->ifc[l + 1];
            const int base = v.nTFP + v.nIE;
            for (int t = 0; t < (int)I.tf_coarse.size(); t++) v.tag[I.tf_coarse[t]] = base + t;
        }
        for (long long idx = 0; idx < v.N; idx++)
            if (v.tag[idx] == TAG_BULK && v.cls[idx] != LBM_NODE_BULK)
                return fail(nullptr, LBM_ERR_BAD_DESC, "interface node without a table entry");
    }
    return LBM_OK;
}

constexpr unsigned long long kWaitLimitNs = 2000000000ull;  // bounded device waits: 2 s
// interface launches with at least this many nodes take one node per thread (enough
// threads to fill 152 SMs); smaller ones take a W-lane segment per node
constexpr int kNodeMin = 32768;
constexpr int T2X = 32, T2YT = 8, T2NR = 2;  // D2Q9 tile: 32 x 8 threads, 2 rows per thread
constexpr int T2Y = T2YT * T2NR;

// D2Q9 bulk tile shapes the autotuner chooses from: threads (TX x TYT), NR rows per thread
struct TileCfg {
    int tx, tyt, nr;
};
constexpr TileCfg kTileCfgs[LBM_TILE_CONFIGS] = {{32, 8, 2}, {32, 4, 4}, {32, 8, 1}, {64, 4, 2}, {32, 16, 1}};
constexpr int T3X = 32, T3Y = 8;   // D3Q19: 32 x 8 columns marching in z (k_bulk3d)
// D3Q19 z chunking the autotuner chooses from: target CTA waves per launch (a chunk of
// fewer planes gives more CTAs; every chunk re-stages two planes)
constexpr int kWaves3[LBM_TILE_CONFIGS] = {4, 2, 8, 1, 16};

void build_tiles(lbm_h h)
{
    const int TX = h->D == 2 ? T2X : T3X, TY = h->D == 2 ? T2Y : T3Y, TZ = 1;
    for (int l = 0; l < h->nl; l++) {
        Level &v = h->lev[l];
        v.tiles[0] = (int)((v.n[0] + TX - 1) / TX);
        v.tiles[1] = (int)((v.n[1] + TY - 1) / TY);
        v.tiles[2] = 1;
        if (h->D == 3) continue;  // 3-D columns are classified plane by plane (check_planes); chunks: plan_chunks
        const long long nt = (long long)v.tiles[0] * v.tiles[1] * v.tiles[2];
        v.tile_flag.assign(nt, TILE_GENERAL);
        const int rz = h->D == 3 ? 2 : 0;
        for (long long t = 0; t < nt; t++) {
            const int bx = (int)(t % v.tiles[0]), by = (int)((t / v.tiles[0]) % v.tiles[1]), bz = (int)(t / ((long long)v.tiles[0] * v.tiles[1]));
            const int64_t x0 = (int64_t)bx * TX, y0 = (int64_t)by * TY, z0 = (int64_t)bz * TZ;
            bool any_node = false;
            for (int64_t z = z0; z < std::min<int64_t>(z0 + TZ, v.n[2]); z++)
                for (int64_t y = y0; y < std::min<int64_t>(y0 + TY, v.n[1]); y++)
                    for (int64_t x = x0; x < std::min<int64_t>(x0 + TX, v.n[0]); x++)
                        if (v.cls[x + v.n[0] * (y + v.n[1] * z)] != LBM_NODE_HOLE) any_node = true;
            if (!any_node) {
                v.tile_flag[t] = TILE_SKIP;
                continue;
            }
            bool fast = x0 - 2 >= 0 && x0 + TX + 2 <= v.n[0] && y0 - 2 >= 0 && y0 + TY + 2 <= v.n[1] &&
                        (h->D == 2 || (z0 - 2 >= 0 && z0 + TZ + 2 <= v.n[2]));
            for (int64_t z = z0 - rz; fast && z < z0 + TZ + rz; z++)
                for (int64_t y = y0 - 2; fast && y < y0 + TY + 2; y++)
                    for (int64_t x = x0 - 2; fast && x < x0 + TX + 2; x++)
                        if (v.cls[x + v.n[0] * (y + v.n[1] * z)] != LBM_NODE_BULK) fast = false;
            v.tile_flag[t] = fast ? TILE_FAST : TILE_GENERAL;
        }
    }
}

// the kernel's geometric tile rule (tile_class), replayed on the host
void tile_bounds(const lbm_h h, int l, int *fast_lo, int *fast_hi, int *child_lo, int *child_hi, int *child_per)
{
    const Level &v = h->lev[l];
    for (int a = 0; a < 3; a++) {
        const bool outline = l > 0 && !v.per[a] && a < h->D;
        fast_lo[a] = outline ? 1 : 0;
        fast_hi[a] = (int)(outline ? v.n[a] - 2 : v.n[a] - 1);
        child_lo[a] = (int)(v.child_lo[a] - v.off[a]);
        child_hi[a] = (int)(v.child_hi[a] - v.off[a]);
        child_per[a] = v.child_per[a];
    }
}

unsigned char geometric_class(const lbm_h h, int l, const int *t0, const int *T)
{
    const Level &v = h->lev[l];
    int flo[3], fhi[3], clo[3], chi[3], cper[3];
    tile_bounds(h, l, flo, fhi, clo, chi, cper);
    bool fast = true;
    for (int a = 0; a < h->D; a++)
        if (t0[a] - 2 < flo[a] || t0[a] + T[a] + 1 > fhi[a]) fast = false;
    if (v.has_child) {
        bool disjoint = false, in_hole = true;
        for (int a = 0; a < h->D; a++) {
            if (cper[a]) continue;
            if (t0[a] + T[a] + 1 < clo[a] || t0[a] - 2 > chi[a]) disjoint = true;
            const int last = std::min<int>(t0[a] + T[a] - 1, (int)v.n[a] - 1);
            if (!(t0[a] > clo[a] && last < chi[a])) in_hole = false;
        }
        if (in_hole) return TILE_SKIP;
        if (!disjoint) fast = false;
    }
    return fast ? TILE_FAST : TILE_GENERAL;
}

// 3-D: the kernel's per-plane rule (plane_class), replayed on the host
int geometric_plane_class(const lbm_h h, int l, int X0, int Y0, int TX, int TY, int p)
{
    const Level &v = h->lev[l];
    int flo[3], fhi[3], clo[3], chi[3], cper[3];
    tile_bounds(h, l, flo, fhi, clo, chi, cper);
    const int lo[3] = {X0 - 2, Y0 - 2, p - 1}, hi[3] = {X0 + TX + 1, Y0 + TY + 1, p + 1};
    bool fast = true;
    for (int a = 0; a < 3; a++)
        if (lo[a] < flo[a] || hi[a] > fhi[a]) fast = false;
    if (v.has_child) {
        bool disjoint = false, in_hole = true;
        const int hlo[3] = {X0 - 1, Y0 - 1, p};
        const int hhi[3] = {std::min<int>(X0 + TX, (int)v.n[0] - 1), std::min<int>(Y0 + TY, (int)v.n[1] - 1), p};
        for (int a = 0; a < 3; a++) {
            if (cper[a]) continue;
            if (hi[a] < clo[a] || lo[a] > chi[a]) disjoint = true;
            if (!(hlo[a] > clo[a] && hhi[a] < chi[a])) in_hole = false;
        }
        if (in_hole) return 1;
        if (!disjoint) fast = false;
    }
    return fast ? 0 : 2;
}

// every (column, plane) of a 3-D level: a fast plane must only meet bulk nodes, a hole
// plane only hole nodes (general planes are correct for any classification)
int check_planes(lbm_h h)
{
    for (int l = 0; l < h->nl; l++) {
        const Level &v = h->lev[l];
        const int tx = (int)((v.n[0] + T3X - 1) / T3X), ty = (int)((v.n[1] + T3Y - 1) / T3Y);
        for (int by = 0; by < ty; by++)
            for (int bx = 0; bx < tx; bx++)
                for (int p = 0; p < (int)v.n[2]; p++) {
                    const int X0 = bx * T3X, Y0 = by * T3Y;
                    const int cls = geometric_plane_class(h, l, X0, Y0, T3X, T3Y, p);
                    if (cls == 2) continue;
                    const int r = cls == 0 ? 2 : 1, rz = cls == 0 ? 1 : 0;
                    for (int z = p - rz; z <= p + rz; z++)
                        for (int y = Y0 - r; y < Y0 + T3Y + r; y++)
                            for (int x = X0 - r; x < X0 + T3X + r; x++) {
                                const bool in = x >= 0 && y >= 0 && z >= 0 && x < v.n[0] && y < v.n[1] && z < v.n[2];
                                if (cls == 0 && (!in || v.cls[x + v.n[0] * (y + v.n[1] * (long long)z)] != LBM_NODE_BULK))
                                    return fail(nullptr, LBM_ERR_BAD_DESC, "internal: fast plane %d of level %d meets a non-bulk node", p, l);
                                if (cls == 1 && in && v.cls[x + v.n[0] * (y + v.n[1] * (long long)z)] != LBM_NODE_HOLE)
                                    return fail(nullptr, LBM_ERR_BAD_DESC, "internal: hole plane %d of level %d meets a node", p, l);
                            }
                }
    }
    return LBM_OK;
}

// every tile: the geometric rule must agree with the node-by-node classification
int check_tiles(lbm_h h)
{
    if (h->D == 3) return check_planes(h);
    for (int c = 0; c < LBM_TILE_CONFIGS; c++) {
        const int TX = kTileCfgs[c].tx, TY = kTileCfgs[c].tyt * kTileCfgs[c].nr;
        const int T[3] = {TX, TY, 1};
        for (int l = 0; l < h->nl; l++) {
            const Level &v = h->lev[l];
            const int tx = (int)((v.n[0] + TX - 1) / TX), ty = (int)((v.n[1] + TY - 1) / TY);
            if (v.use_tflag) h->lev[l].tflag[c].assign((size_t)tx * ty, TILE_GENERAL);
            for (int by = 0; by < ty; by++)
                for (int bx = 0; bx < tx; bx++) {
                    const int x0 = bx * TX, y0 = by * TY;
                    const int t0[3] = {x0, y0, 0};
                    // node-by-node class of this tile
                    bool any = false, fast = x0 - 2 >= 0 && x0 + TX + 2 <= v.n[0] && y0 - 2 >= 0 && y0 + TY + 2 <= v.n[1];
                    for (int64_t y = y0; y < std::min<int64_t>(y0 + TY, v.n[1]); y++)
                        for (int64_t x = x0; x < std::min<int64_t>(x0 + TX, v.n[0]); x++)
                            any = any || v.cls[x + v.n[0] * y] != LBM_NODE_HOLE;
                    for (int64_t y = y0 - 2; fast && y < y0 + TY + 2; y++)
                        for (int64_t x = x0 - 2; fast && x < x0 + TX + 2; x++)
                            fast = v.cls[x + v.n[0] * y] == LBM_NODE_BULK;
                    const unsigned char want = !any ? TILE_SKIP : (fast ? TILE_FAST : TILE_GENERAL);
                    if (v.use_tflag) {
                        h->lev[l].tflag[c][(size_t)bx + (size_t)tx * by] = want;
                        continue;
                    }
                    if (geometric_class(h, l, t0, T) != want)
                        return fail(nullptr, LBM_ERR_BAD_DESC, "internal: tile (%d,%d) of level %d, shape %d, "
                                    "classified inconsistently", bx, by, l, c);
                }
        }
    }
    return LBM_OK;
}

// dual-cell volume of every node restricted to its level's region, in level-0 cell units
std::vector<double> node_weights(const lbm_h h, int l)
{
    const Level &v = h->lev[l];
    std::vector<double> w(v.N, 0.0);
    const double base = std::ldexp(1.0, -h->D * l);
    if (v.use_tflag) {
        // staircase regions: the node's dual cell in 2^D quarters, one per level-l cell
        // around it; a quarter counts when its cell lies in the level's region and not in
        // the child's
        const double q = std::ldexp(1.0, -h->D);
        for (long long idx = 0; idx < v.N; idx++) {
            if (v.cls[idx] == LBM_NODE_HOLE) continue;
            int64_t p[3];
            global_of(v, idx, p);
            double acc = 0.0;
            for (int k = 0; k < (1 << h->D); k++) {
                int64_t c[3] = {p[0], p[1], p[2]};
                for (int a = 0; a < h->D; a++) c[a] -= (k >> a) & 1;
                int64_t cp[3] = {0, 0, 0};  // parent cell holding level-l cell c
                for (int a = 0; a < h->D; a++) cp[a] = c[a] >= 0 ? c[a] / 2 : -((1 - c[a]) / 2);
                const bool own = l == 0 || refines(h, l, cp);
                const bool child = l + 1 < h->nl && refines(h, l + 1, c);
                if (own && !child) acc += q;
            }
            w[idx] = base * acc;
        }
        return w;
    }
    for (long long idx = 0; idx < v.N; idx++) {
        if (v.cls[idx] == LBM_NODE_HOLE) continue;
        int64_t p[3];
        global_of(v, idx, p);
        double own = 1.0, child = v.has_child ? 1.0 : 0.0;
        for (int a = 0; a < h->D; a++) {
            const int64_t q = p[a] - v.off[a];
            if (!v.per[a] && (q == 0 || q == v.n[a] - 1)) own *= 0.5;
            if (v.has_child && !v.child_per[a]) {
                if (p[a] < v.child_lo[a] || p[a] > v.child_hi[a]) child = 0.0;
                else if (p[a] == v.child_lo[a] || p[a] == v.child_hi[a]) child *= 0.5;
            }
        }
        w[idx] = base * (own - child);
    }
    return w;
}

// ------------------------------------------------------------------ bulk tensor copies (D3Q19)
using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encode_tiled()
{
    static std::once_flag once;
    static EncodeTiled fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiled)p;
    });
    return fn;
}

// dynamic shared memory limit of the 3-D kernel for storage S; CTAs per SM
template <typename S>
int bulk3d_prepare(int *per_sm)
{
    using G = Stage3<19, S, T3X, T3Y>;
    auto kern = k_bulk3d<19, S, T3X, T3Y, false>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::smem_bytes) != cudaSuccess)
        return -1;
    if constexpr (std::is_same<S, __half>::value) {
        if (cudaFuncSetAttribute(k_bulk3d<19, S, T3X, T3Y, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)G::smem_bytes) != cudaSuccess)
            return -1;
    }
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, kern, T3X * T3Y, G::smem_bytes) != cudaSuccess) return -1;
    return 0;
}

// z chunk of a 3-D level: about kWaves3[cfg] waves of CTAs, chunks of at least 8 planes
int plan_chunks(lbm_h h, int l)
{
    Level &v = h->lev[l];
    int dev = 0, sms = 0, per_sm = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int st = h->d.storage;
    const int rc = st == LBM_F64 ? bulk3d_prepare<double>(&per_sm)
                   : st == LBM_F32 ? bulk3d_prepare<float>(&per_sm)
                                   : bulk3d_prepare<__half>(&per_sm);
    if (rc != 0 || per_sm < 1) return fail(h, LBM_ERR_CUDA, "3-D bulk kernel does not fit an SM");
    const long long cols = (long long)v.tiles[0] * v.tiles[1];
    const long long want = (long long)kWaves3[v.tile_cfg] * sms * per_sm;
    const long long nmax = std::max<long long>(1, v.n[2] / 8);
    const long long nch = std::min<long long>(std::max<long long>(1, (want + cols - 1) / cols), nmax);
    v.zc = (int)((v.n[2] + nch - 1) / nch);
    v.tiles[2] = (int)((v.n[2] + v.zc - 1) / v.zc);
    return LBM_OK;
}

// 4-D maps (x, y, z, population) of both population buffers of a 3-D level; the box is
// TX + 2 XA x TY + 4 nodes of one plane (Stage3) and 1, 2, 4 or 5 consecutive
// populations (one map per depth: a run of populations with the same c_z is one copy)
int make_tensor_maps(lbm_h h, int l)
{
    Level &v = h->lev[l];
    EncodeTiled enc = encode_tiled();
    if (!enc) return fail(h, LBM_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
    const int st = h->d.storage;
    const size_t es = store_size(st);
    const int xa = 16 / (int)es;
    const CUtensorMapDataType dt = st == LBM_F64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                                   : st == LBM_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                                   : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
    const cuuint64_t dims[4] = {(cuuint64_t)v.n[0], (cuuint64_t)v.n[1], (cuuint64_t)v.n[2], (cuuint64_t)h->Q};
    const cuuint64_t strides[3] = {(cuuint64_t)(v.px * es), (cuuint64_t)(v.px * v.n[1] * es), (cuuint64_t)(v.pitch * es)};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    for (int k = 0; k < 2; k++)
        for (int m = 0; m < 4; m++) {
            const cuuint32_t box[4] = {(cuuint32_t)(T3X + 2 * xa), (cuuint32_t)(T3Y + 4), 1, (cuuint32_t)kDepths[m]};
            const CUresult r = enc(&v.tmap[k].m[m], dt, 4, v.f[k], dims, strides, box, estr,
                                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS)
                return fail(h, LBM_ERR_CUDA, "tensor map of level %d buffer %d (driver error %d)", l, k, (int)r);
        }
    return LBM_OK;
}

int upload_all(lbm_h h)
{
    bool ok = true;
    const size_t ss = store_size(h->d.storage);
    const int Q = h->Q;
    for (int l = 0; l < h->nl; l++) {
        Level &v = h->lev[l];
        for (int k = 0; k < 2; k++) {
            v.f[k] = dev_alloc(h, (size_t)Q * v.pitch * ss);
            if (!v.f[k]) return fail(h, LBM_ERR_OOM, "population buffer of level %d (%zu bytes)", l, (size_t)Q * v.pitch * ss);
        }
        {
            // device tag map in the padded slot layout
            std::vector<int> slot_tag((size_t)v.NS, TAG_HOLE);
            for (long long idx = 0; idx < v.N; idx++) {
                const long long x = idx % v.n[0], yz = idx / v.n[0];
                slot_tag[(size_t)(x + v.px * yz)] = v.tag[(size_t)idx];
            }
            v.d_tag = upload(h, slot_tag, &ok);
        }
        if (h->D == 3) {
            int rc = make_tensor_maps(h, l);
            if (rc == LBM_OK) rc = plan_chunks(h, l);
            if (rc != LBM_OK) return rc;
        }
        const size_t ni = std::max(1, v.nif), as = arith_size(h->d.storage);
        v.if_pop = dev_alloc(h, ni * Q * as);
        v.if_mac = dev_alloc(h, ni * 4 * as);
        v.if_S = dev_alloc(h, ni * 6 * as);
        v.if_C = dev_alloc(h, ni * 6 * as);
        v.d_wnode = upload(h, node_weights(h, l), &ok);
        if (v.use_tflag)
            for (int c = 0; c < LBM_TILE_CONFIGS; c++) v.d_tflag[c] = upload(h, v.tflag[c], &ok);
        if (!ok || !v.if_pop || !v.if_mac || !v.if_S || !v.if_C) return fail(h, LBM_ERR_OOM, "tables of level %d", l);
        CK(cudaMemset(v.if_pop, 0, ni * Q * as));
        CK(cudaMemset(v.if_mac, 0, ni * 4 * as));
        CK(cudaMemset(v.if_S, 0, ni * 6 * as));
        CK(cudaMemset(v.if_C, 0, ni * 6 * as));
    }
    for (int l = 1; l < h->nl; l++) {
        Iface &I = h->ifc[l];
        IfaceDev &g = I.dev;
        g.nTF = (int)I.tf_fine.size();
        g.nIE = (int)I.ie_fine.size();
        g.nRing = (int)I.ring_coarse.size();
        g.tf_f = upload(h, coords3(h->lev[l], I.tf_fine), &ok);
        g.tf_c = upload(h, coords3(h->lev[l - 1], I.tf_coarse), &ok);
        g.tf_kf = upload(h, I.tf_kf, &ok);
        g.tf_kc = upload(h, I.tf_kc, &ok);
        g.tf_gc = upload(h, I.tf_gc, &ok);
        g.tf_rkind = upload(h, I.tf_rkind, &ok);
        g.tf_ridx = upload(h, I.tf_ridx, &ok);
        g.ie_f = upload(h, coords3(h->lev[l], I.ie_fine), &ok);
        g.ie_kf = upload(h, I.ie_kf, &ok);
        g.ie_nst = upload(h, I.ie_nst, &ok);
        g.ie_st = upload(h, I.ie_st, &ok);
        if (h->d.storage == LBM_F64) {
            g.ie_w = upload(h, I.ie_w, &ok);
        } else {
            const std::vector<float> w32(I.ie_w.begin(), I.ie_w.end());  // Lagrange weights: exact in FP32
            for (size_t k = 0; k < w32.size(); k++)
                if ((double)w32[k] != I.ie_w[k]) return fail(h, LBM_ERR_BAD_DESC, "internal: stencil weight not exact in FP32");
            g.ie_w = upload(h, w32, &ok);
        }
        g.ring_c = upload(h, coords3(h->lev[l - 1], I.ring_coarse), &ok);
        g.hist_f = dev_alloc(h, (size_t)3 * Q * std::max(1, g.nTF) * arith_size(h->d.storage));
        g.hist_m = dev_alloc(h, (size_t)3 * 4 * std::max(1, g.nRing) * arith_size(h->d.storage));
        g.tfc_base = h->lev[l - 1].nTFP + h->lev[l - 1].nIE;
        g.R = I.R;
        g.Rf = (float)I.R;
        g.Rinv = 1.0 / I.R;
        if (!ok || !g.hist_f || !g.hist_m) return fail(h, LBM_ERR_OOM, "interface %d tables", l);
    }
    h->d_status = (int *)dev_alloc(h, 2 * sizeof(int));
    if (!h->d_status) return fail(h, LBM_ERR_OOM, "status word");
    h->d_maxit = h->d_status + 1;
    CK(cudaMemset(h->d_status, 0, 2 * sizeof(int)));
    h->red_blocks = 304;
    h->d_partial = (double *)dev_alloc(h, (size_t)h->red_blocks * 4 * sizeof(double) + 4 * sizeof(double));
    if (!h->d_partial) return fail(h, LBM_ERR_OOM, "reduction scratch");
    h->d_red = h->d_partial + (size_t)h->red_blocks * 4;
    return LBM_OK;
}

LevelDev level_dev(const lbm_h h, int l)
{
    const Level &v = h->lev[l];
    LevelDev d{};
    for (int a = 0; a < 3; a++) {
        d.g.n[a] = (int)v.n[a];
        d.g.per[a] = v.per[a];
        d.tiles[a] = v.tiles[a];
    }
    d.g.N = v.N;
    d.g.px = (int)v.px;
    for (int i = 0; i < 19; i++) d.g.shift[i] = h->shift[i];
    d.g.NS = v.NS;
    d.g.pitch = v.pitch;
    d.f[0] = v.f[0];
    d.f[1] = v.f[1];
    d.tag = v.d_tag;
    d.if_pop = v.if_pop;
    d.if_mac = v.if_mac;
    d.if_S = v.if_S;
    d.if_C = v.if_C;
    d.nif = std::max(1, v.nif);
    d.tau = v.tau;
    d.om = 1.0 - 1.0 / v.tau;
    d.sigma = h->d.sigma;
    d.spsi = (double)h->d.psi_sign;
    // FP16 shift folded into the D3Q19 bulk kernel's moments and pair outputs
    if (h->Q == 19) {
        double sm[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
        for (int i = 0; i < 19; i++) {
            const double si = (double)h->shift[i];
            const int c0 = Lat<19>::c(i, 0), c1 = Lat<19>::c(i, 1), c2 = Lat<19>::c(i, 2);
            sm[0] += si;
            sm[1] += c0 * si;
            sm[2] += c1 * si;
            sm[3] += c2 * si;
            sm[4] += c0 * c0 * si;
            sm[5] += c1 * c1 * si;
            sm[6] += c2 * c2 * si;
            sm[7] += c0 * c1 * si;
            sm[8] += c0 * c2 * si;
            sm[9] += c1 * c2 * si;
        }
        for (int q = 0; q < 10; q++) d.smom[q] = (float)sm[q];
        d.she[0] = (float)((double)h->shift[0] / Lat<19>::w(0));
        d.sho[0] = 0.0f;
        for (int i = 1; i < 19; i += 2) {
            const double w = Lat<19>::w(i), sa = h->shift[i], sb = h->shift[i + 1];
            d.she[i] = (float)((sa + sb) / (2.0 * w));
            d.sho[i] = (float)((sa - sb) / (2.0 * w));
            d.she[i + 1] = d.she[i];
            d.sho[i + 1] = -d.sho[i];
        }
    }
    d.tauf = (float)d.tau;
    d.omf = (float)d.om;
    d.sigmaf = (float)d.sigma;
    d.spsif = (float)d.spsi;
    tile_bounds(h, l, d.fast_lo, d.fast_hi, d.child_lo, d.child_hi, d.child_per);
    d.has_child = v.has_child ? 1 : 0;
    d.tile_flags = (h->D == 2 && v.use_tflag) ? v.d_tflag[v.tile_cfg] : nullptr;
    d.ie_base = v.nTFP;
    d.n_ie = v.nIE;
    if (l > 0) {
        d.ie_nst = h->ifc[l].dev.ie_nst;
        d.ie_st = h->ifc[l].dev.ie_st;
        d.ie_w = h->ifc[l].dev.ie_w;
    }
    return d;
}

// ------------------------------------------------------------------ schedule
// a launch that may start while the previous kernel of its stream finishes (the
// kernel waits for that kernel's completion before touching memory: pdl_enter)
template <typename... KArgs, typename... Args>
void launch_chained(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, Args &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

template <int Q, typename S, int TX, int TYT, int NR>
void launch_bulk2d_cfg(lbm_h h, int l, const void *src, void *dst, typename St<S>::R tau, typename St<S>::R om,
                       typename St<S>::R sig, typename St<S>::R sps, cudaStream_t st)
{
    const Level &v = h->lev[l];
    const dim3 grid((unsigned)((v.n[0] + TX - 1) / TX), (unsigned)((v.n[1] + TYT * NR - 1) / (TYT * NR)), 1);
    launch_chained(k_bulk2d<Q, S, TX, TYT, NR>, grid, dim3(TX * TYT), 0, st, level_dev(h, l), (const S *)src, (S *)dst,
                   tau, om, sig, sps);
}

template <int Q, typename S>
void launch_bulk2d(lbm_h h, int l, int cfg, const void *src, void *dst, typename St<S>::R tau,
                   typename St<S>::R om, typename St<S>::R sig, typename St<S>::R sps, cudaStream_t st)
{
    switch (cfg) {
    case 1: launch_bulk2d_cfg<Q, S, 32, 4, 4>(h, l, src, dst, tau, om, sig, sps, st); break;
    case 2: launch_bulk2d_cfg<Q, S, 32, 8, 1>(h, l, src, dst, tau, om, sig, sps, st); break;
    case 3: launch_bulk2d_cfg<Q, S, 64, 4, 2>(h, l, src, dst, tau, om, sig, sps, st); break;
    case 4: launch_bulk2d_cfg<Q, S, 32, 16, 1>(h, l, src, dst, tau, om, sig, sps, st); break;
    default: launch_bulk2d_cfg<Q, S, 32, 8, 2>(h, l, src, dst, tau, om, sig, sps, st); break;
    }
}

// one node per thread (true) or one W-lane segment per node for an interface launch of n nodes
bool node_mapping(const lbm_h h, int n)
{
    if (h->if_mode == LBM_IFACE_NODE) return true;
    if (h->if_mode == LBM_IFACE_SEGMENT) return false;
    return n >= kNodeMin;
}

template <int Q, typename S>
struct Sched {
    static void bulk(lbm_h h, int l, const void *src, void *dst, cudaStream_t stream = nullptr)
    {
        const cudaStream_t st = stream ? stream : h->stream;
        const Level &v = h->lev[l];
        const dim3 nt(v.tiles[0], v.tiles[1], v.tiles[2]);
        const double spsi = (double)h->d.psi_sign;
        int ev = -1;
        if (h->timing) {
            ev = (int)h->ev_pairs.size() * 2;
            while ((int)h->ev_pool.size() < ev + 2) {
                cudaEvent_t e;
                cudaEventCreate(&e);
                h->ev_pool.push_back(e);
            }
            cudaEventRecord(h->ev_pool[ev], h->stream);
        }
        using R = typename St<S>::R;
        const R tau = (R)v.tau, om = (R)(1.0 - 1.0 / v.tau), sig = (R)h->d.sigma, sps = (R)spsi;
        if constexpr (Lat<Q>::D == 2)
            launch_bulk2d<Q, S>(h, l, v.tile_cfg, src, dst, tau, om, sig, sps, st);
        else {
            auto k3 = k_bulk3d<Q, S, T3X, T3Y, false>;
            if constexpr (std::is_same<S, __half>::value)
                if (h->plain_shift) k3 = k_bulk3d<Q, S, T3X, T3Y, true>;
            launch_chained(k3, nt, dim3(T3X * T3Y), Stage3<Q, S, T3X, T3Y>::smem_bytes, st,
                           v.tmap[src == v.f[0] ? 0 : 1], level_dev(h, l), (const S *)src, (S *)dst, tau, om, sig,
                           sps, v.zc, h->d_status, h->withhold_level == l ? h->withhold_limit_ns : kWaitLimitNs,
                           h->withhold_level == l ? h->withhold_block : -1, h->withhold_level == l ? h->withhold_k : -1);
        }
        h->launch_counter++;
        if (h->timing) {
            cudaEventRecord(h->ev_pool[ev + 1], h->stream);
            h->ev_pairs.push_back({l, ev});
        }
    }

    static TimeW weights(int phase, long long kp) { return time_weights(phase, kp); }

    // one step of level l (Sec. 3.5): k is the level's step index, kp its parent's
    static void level_step(lbm_h h, int l, long long k, int phase, long long kp)
    {
        NvtxRange range(kLevelRange[l]);
        Level &v = h->lev[l];
        const void *fA = v.f[k & 1];
        void *fB = v.f[(k + 1) & 1];
        // interface kernels, 128 threads per block: one node per thread when a launch has
        // at least kNodeMin nodes (throughput), else one W-lane segment per node (latency)
        constexpr int W = Q <= 16 ? 16 : 32;
        auto per_block = [h](int n) { return node_mapping(h, n) ? 128 : 128 / W; };
        LevelDev dv = level_dev(h, l);
        // Newton at this level's TF nodes and the history push for the child interface
        // are independent: one launch
        const bool recon = l > 0 && h->ifc[l].dev.nTF > 0;
        const bool hist = l + 1 < h->nl && h->ifc[l + 1].dev.nTF + h->ifc[l + 1].dev.nRing > 0;
        TimeW tw{};
        if (l > 0) tw = weights(phase, kp);
        if (recon || hist) {
            const IfaceDev Ir = recon ? h->ifc[l].dev : IfaceDev{};
            const IfaceDev Ih = hist ? h->ifc[l + 1].dev : IfaceDev{};
            const int nr = recon ? Ir.nTF : 0, nh = hist ? Ih.nTF + Ih.nRing : 0;
            const int per = per_block(nr + nh);
            const int nbr = (nr + per - 1) / per, nbh = (nh + per - 1) / per;
            const LevelDev dc = l > 0 ? level_dev(h, l - 1) : dv;
            launch_chained(per == 128 ? k_recon_hist<Q, S, true> : k_recon_hist<Q, S, false>, dim3(nbr + nbh), dim3(128),
                           0, h->stream, Ir, dv, dc, (const S *)fA, tw, phase, h->d_status, h->d_maxit, nbr, Ih, dv.g,
                           (const S *)fA, (int)((k + 1) % 3));
            h->launch_counter++;
        }
        // TF gradients and hanging nodes of this level read this level's populations, TF
        // rows and ring history and write this level's TF and hanging rows; the child
        // level's sub-steps touch only the child's data, the history of the child
        // interface and this level's child-TF rows.  So with a child the launch runs on
        // the side stream beside the child's sub-steps; the bulk launch joins both.
        bool forked = false;
        if (l > 0) {
            const IfaceDev &I = h->ifc[l].dev;
            const int per = per_block(I.nTF + I.nIE);
            const int nbg = (I.nTF + per - 1) / per, nbi = (I.nIE + per - 1) / per;
            if (nbg + nbi > 0) {
                cudaStream_t st = h->stream;
                if (l + 1 < h->nl) {
                    cudaEventRecord(h->ev_fork[l], h->stream);
                    cudaStreamWaitEvent(h->side, h->ev_fork[l], 0);
                    st = h->side;
                    forked = true;
                }
                launch_chained(per == 128 ? k_grad_ie<Q, S, true> : k_grad_ie<Q, S, false>, dim3(nbg + nbi), dim3(128), 0,
                               st, I, dv, level_dev(h, l - 1), (const S *)fA, tw, phase, nbg);
                h->launch_counter++;
                if (Lat<Q>::D == 3 && dv.n_ie > 0) {
                    // S and C of the hanging nodes from the TF rows just written (the 3-D
                    // bulk kernel reads them as table rows)
                    launch_chained(k_ie_sc<typename St<S>::R>, dim3((dv.n_ie + 127) / 128), dim3(128), 0, st, dv);
                    h->launch_counter++;
                }
                if (forked) cudaEventRecord(h->ev_join[l], h->side);
            }
        }
        // a sync sub-step has now issued everything that writes the parent's child-TF
        // rows (the coarse rebuild in the Newton launch, S and C in the gradient launch)
        if (l > 0 && phase == 1) cudaEventRecord(h->ev_parent[l], forked ? h->side : h->stream);
        if (l + 1 < h->nl) {
            level_step(h, l + 1, 2 * k, 0, k);
            level_step(h, l + 1, 2 * k + 1, 1, k);
        }
        if (l + 1 < h->nl && !h->timing) {
            // this level's bulk launch beside the rest of the child's sync sub-step; the
            // main stream joins it before anything can read this level's new state
            cudaStreamWaitEvent(h->side2[l], h->ev_parent[l + 1], 0);
            if (forked) cudaStreamWaitEvent(h->side2[l], h->ev_join[l], 0);
            bulk(h, l, fA, fB, h->side2[l]);
            cudaEventRecord(h->ev_bulk[l], h->side2[l]);
            cudaStreamWaitEvent(h->stream, h->ev_bulk[l], 0);
        } else {
            if (forked) cudaStreamWaitEvent(h->stream, h->ev_join[l], 0);
            bulk(h, l, fA, fB);
        }
    }

    static void coarse_step(lbm_h h, long long n) { level_step(h, 0, n, 1, -1); }

    static int init_level(lbm_h h, int l, const double *rho, const double *u)
    {
        Level &v = h->lev[l];
        LevelDev dv = level_dev(h, l);
        const int B = 256;
        k_init<Q, S><<<(unsigned)((v.N + B - 1) / B), B, 0, h->stream>>>(dv.g, v.d_tag, rho, u, (S *)v.f[0],
                                                                           (S *)v.f[1]);
        if (l + 1 < h->nl) {
            const IfaceDev &I = h->ifc[l + 1].dev;
            const int n = I.nTF + I.nRing;
            constexpr int SEG = 128;  // nodes per block
            if (n > 0) k_hist<Q, S><<<(n + SEG - 1) / SEG, 128, 0, h->stream>>>(I, dv.g, (const S *)v.f[0], 0, 1);
        }
        return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
    }

    static void macros(lbm_h h, int l, double *rho, double *u, double *pops)
    {
        Level &v = h->lev[l];
        const long long k = h->ncoarse << l;
        LevelDev dv = level_dev(h, l);
        const int B = 256;
        k_macros<Q, S><<<(unsigned)((v.N + B - 1) / B), B, 0, h->stream>>>(dv.g, v.d_tag, (const S *)v.f[k & 1],
                                                                             rho, u, pops);
    }

    static void probe(lbm_h h, const long long *kstep, int row, int n)
    {
        k_probe<Q, S><<<(n + 63) / 64, 64, 0, h->stream>>>(h->probes, h->d_levs, kstep, row);
    }

    static void reduce(lbm_h h, int l)
    {
        Level &v = h->lev[l];
        const long long k = h->ncoarse << l;
        LevelDev dv = level_dev(h, l);
        k_reduce_partial<Q, S><<<h->red_blocks, 256, 0, h->stream>>>(dv.g, v.d_tag, (const S *)v.f[k & 1], v.d_wnode,
                                                                      h->d_partial, h->d_status);
        k_reduce_final<<<1, 256, 0, h->stream>>>(h->d_partial, h->red_blocks, h->d_red);
    }
};

template <typename Fn>
void dispatch(lbm_h h, Fn &&fn)
{
    if (h->Q == 9) {
        if (h->d.storage == LBM_F64) fn(Sched<9, double>());
        else if (h->d.storage == LBM_F32) fn(Sched<9, float>());
        else fn(Sched<9, __half>());
    } else {
        if (h->d.storage == LBM_F64) fn(Sched<19, double>());
        else if (h->d.storage == LBM_F32) fn(Sched<19, float>());
        else fn(Sched<19, __half>());
    }
}

int issue_coarse_step(lbm_h h, long long n)
{
    h->launch_counter = 0;
    dispatch(h, [&](auto s) { decltype(s)::coarse_step(h, n); });
    h->launches += h->launch_counter;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(h, LBM_ERR_CUDA, "launch: %s", cudaGetErrorString(e));
    return LBM_OK;
}

int run_graph(lbm_h h, long long n)
{
    const int key = (int)(n % 6);
    auto it = h->graphs.find(key);
    if (it == h->graphs.end()) {
        cudaGraph_t g;
        CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
        h->launch_counter = 0;
        dispatch(h, [&](auto s) { decltype(s)::coarse_step(h, n); });
        const int64_t cnt = h->launch_counter;
        CK(cudaStreamEndCapture(h->stream, &g));
        cudaGraphExec_t ge;
        CK(cudaGraphInstantiate(&ge, g, 0));
        cudaGraphDestroy(g);
        it = h->graphs.emplace(key, ge).first;
        h->graph_launches[key] = cnt;
    }
    CK(cudaGraphLaunch(it->second, h->stream));
    h->launches += h->graph_launches[key];
    return LBM_OK;
}

bool check_level(lbm_h h, int level)
{
    if (!h) return false;
    if (level < 0 || level >= h->nl) {
        fail(h, LBM_ERR_ARG, "level %d out of range [0,%d)", level, h->nl);
        return false;
    }
    return true;
}

}  // namespace

// ================================================================== C-ABI
extern "C" {

const char *lbm_create_error(void) { return g_create_error.c_str(); }

static int create_impl(const lbm_hierarchy_desc *desc, const uint8_t *const *masks, void *cuda_stream, lbm_h *out);

int lbm_create_hierarchy(const lbm_hierarchy_desc *desc, void *cuda_stream, lbm_h *out)
{
    return create_impl(desc, nullptr, cuda_stream, out);
}

int lbm_create_hierarchy_masked(const lbm_hierarchy_desc *desc, const uint8_t *const *masks, void *cuda_stream,
                                lbm_h *out)
{
    return create_impl(desc, masks, cuda_stream, out);
}

static int create_impl(const lbm_hierarchy_desc *desc, const uint8_t *const *masks, void *cuda_stream, lbm_h *out)
{
    if (!out) return fail(nullptr, LBM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!desc) return fail(nullptr, LBM_ERR_ARG, "desc is NULL");
    if (desc->lattice != 9 && desc->lattice != 19) return fail(nullptr, LBM_ERR_BAD_DESC, "lattice must be 9 or 19");
    if (desc->n_levels < 1 || desc->n_levels > LBM_MAX_LEVELS) return fail(nullptr, LBM_ERR_BAD_DESC, "n_levels out of range");
    if (desc->storage < LBM_F64 || desc->storage > LBM_F16S) return fail(nullptr, LBM_ERR_BAD_DESC, "bad storage");
    if (desc->dc_variant != 1 && desc->dc_variant != 2) return fail(nullptr, LBM_ERR_BAD_DESC, "dc_variant must be 1 or 2");
    if (!(desc->nu0 > 0.0) || !(desc->sigma >= 0.0 && desc->sigma <= 1.0))
        return fail(nullptr, LBM_ERR_BAD_DESC, "nu0 must be > 0 and sigma in [0,1]");
    if ((desc->alloc == nullptr) != (desc->free == nullptr)) return fail(nullptr, LBM_ERR_BAD_DESC, "alloc and free go together");
    const int D = desc->lattice == 9 ? 2 : 3;
    for (int a = 0; a < 3; a++)
        if (!(std::fabs(desc->u_shift[a]) < 0.3) || (a >= D && desc->u_shift[a] != 0.0))
            return fail(nullptr, LBM_ERR_BAD_DESC, "u_shift components must be below 0.3 (0 beyond the lattice's dimension)");
    for (int a = 0; a < 3; a++) {
        if (desc->coarse_n[a] < 1 || desc->coarse_n[a] > (1 << 20)) return fail(nullptr, LBM_ERR_BAD_DESC, "coarse_n out of range");
        if (a >= D && desc->coarse_n[a] != 1) return fail(nullptr, LBM_ERR_BAD_DESC, "coarse_n[2] must be 1 for D2Q9");
        if (a < D && desc->coarse_n[a] < 8) return fail(nullptr, LBM_ERR_BAD_DESC, "coarse_n must be >= 8");
    }
    lbm_h h = new lbm_hierarchy();
    h->d = *desc;
    h->Q = desc->lattice;
    h->D = D;
    h->nl = desc->n_levels;
    for (int i = 0; i < h->Q; i++)  // s_i = f_i^eq(1, u_shift): w_i for u_shift = 0
        h->shift[i] = (float)(h->Q == 9 ? feq_one<9>(i, 1.0, desc->u_shift) : feq_one<19>(i, 1.0, desc->u_shift));
    h->plain_shift = desc->storage == LBM_F16S && desc->u_shift[0] == 0.0 && desc->u_shift[1] == 0.0 &&
                     desc->u_shift[2] == 0.0;
    for (int l = 1; l < h->nl && masks; l++) {
        if (!masks[l]) continue;
        size_t cells = 1;
        const int64_t psc = (int64_t)1 << (l - 1);
        for (int a = 0; a < D; a++) {
            const int64_t e = (desc->box_hi[l][a] - desc->box_lo[l][a]) * psc;
            if (e < 1) {
                delete h;
                return fail(nullptr, LBM_ERR_BAD_DESC, "level %d: empty box for its mask", l);
            }
            cells *= (size_t)e;
        }
        h->mask[l].assign(masks[l], masks[l] + cells);
        h->masked = true;
    }
    int rc = build_geometry(h);
    if (rc == LBM_OK) rc = build_interfaces(h);
    if (rc != LBM_OK) {
        delete h;
        return rc;
    }
    build_tiles(h);
    for (int l = 1; l < h->nl; l++)
        if (!h->mask[l].empty()) h->lev[l].use_tflag = h->lev[l - 1].use_tflag = true;
    rc = check_tiles(h);
    if (rc != LBM_OK) {
        delete h;
        return rc;
    }
    for (int l = 0; l < h->nl; l++)
        if (h->lev[l].N > (long long)2147483647) {
            delete h;
            return fail(nullptr, LBM_ERR_BAD_DESC, "level %d has more than 2^31 box nodes", l);
        }
    if (cudaGetDevice(&h->device) != cudaSuccess) {
        delete h;
        return fail(nullptr, LBM_ERR_CUDA, "cudaGetDevice failed");
    }
    if (cuda_stream) {
        h->stream = (cudaStream_t)cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete h;
            return fail(nullptr, LBM_ERR_CUDA, "cudaStreamCreateWithFlags failed");
        }
        h->own_stream = true;
    }
    bool evok = cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking) == cudaSuccess;
    for (int l = 0; l < LBM_MAX_LEVELS && evok; l++)
        evok = (l + 1 >= h->nl || cudaStreamCreateWithFlags(&h->side2[l], cudaStreamNonBlocking) == cudaSuccess) &&
               cudaEventCreateWithFlags(&h->ev_fork[l], cudaEventDisableTiming) == cudaSuccess &&
               cudaEventCreateWithFlags(&h->ev_join[l], cudaEventDisableTiming) == cudaSuccess &&
               cudaEventCreateWithFlags(&h->ev_parent[l], cudaEventDisableTiming) == cudaSuccess &&
               cudaEventCreateWithFlags(&h->ev_bulk[l], cudaEventDisableTiming) == cudaSuccess;
    if (!evok) {
        g_create_error = "cudaStreamCreateWithFlags / cudaEventCreateWithFlags failed";
        lbm_destroy(h);
        return LBM_ERR_CUDA;
    }
    rc = upload_all(h);
    if (rc != LBM_OK) {
        g_create_error = h->err;
        lbm_destroy(h);
        return rc;
    }
    *out = h;
    return LBM_OK;
}

int lbm_query_level(lbm_h h, int level, int64_t n_out[3], int64_t off_out[3], int64_t *n_active, double *tau_out)
{
    if (!check_level(h, level)) return h ? LBM_ERR_ARG : LBM_ERR_ARG;
    const Level &v = h->lev[level];
    for (int a = 0; a < 3; a++) {
        if (n_out) n_out[a] = v.n[a];
        if (off_out) off_out[a] = v.off[a];
    }
    if (n_active) *n_active = v.n_active;
    if (tau_out) *tau_out = v.tau;
    return LBM_OK;
}

int lbm_node_class(lbm_h h, int level, uint8_t *cls_out)
{
    if (!check_level(h, level)) return LBM_ERR_ARG;
    if (!cls_out) return fail(h, LBM_ERR_ARG, "cls_out is NULL");
    memcpy(cls_out, h->lev[level].cls.data(), h->lev[level].N);
    return LBM_OK;
}

int lbm_init_fields(lbm_h h, int level, const double *rho, const double *u, int on_device)
{
    if (!check_level(h, level)) return LBM_ERR_ARG;
    if (!rho || !u) return fail(h, LBM_ERR_ARG, "rho/u is NULL");
    const Level &v = h->lev[level];
    const double *drho = rho, *du = u;
    double *tmp = nullptr;
    if (!on_device) {
        tmp = (double *)tmp_alloc(h, (size_t)(1 + h->D) * v.N * sizeof(double));
        if (!tmp) return fail(h, LBM_ERR_OOM, "staging buffer");
        CK(cudaMemcpyAsync(tmp, rho, v.N * sizeof(double), cudaMemcpyHostToDevice, h->stream));
        CK(cudaMemcpyAsync(tmp + v.N, u, (size_t)h->D * v.N * sizeof(double), cudaMemcpyHostToDevice, h->stream));
        drho = tmp;
        du = tmp + v.N;
    }
    int rc = LBM_OK;
    dispatch(h, [&](auto s) { rc = decltype(s)::init_level(h, level, drho, du); });
    h->ncoarse = 0;
    if (tmp) {
        CK(cudaStreamSynchronize(h->stream));
        tmp_free(h, tmp);
    }
    if (rc != LBM_OK) return fail(h, rc, "init kernel launch failed");
    return LBM_OK;
}

static int batch_advance(lbm_h h, int64_t n);

// one row of probe samples for the current state (stream-ordered)
static int record_probes(lbm_h h)
{
    std::vector<long long> ks(h->nl);
    for (int l = 0; l < h->nl; l++) ks[l] = h->ncoarse << l;
    CK(cudaMemcpyAsync(h->d_kstep + (size_t)(h->probe_rows % 64) * LBM_MAX_LEVELS, ks.data(), h->nl * sizeof(long long),
                       cudaMemcpyHostToDevice, h->stream));
    const int n = h->probes.n;
    const int row = (int)h->probe_rows;
    const long long *kp = h->d_kstep + (size_t)(h->probe_rows % 64) * LBM_MAX_LEVELS;
    dispatch(h, [&](auto s) {
        using Sc = decltype(s);
        Sc::probe(h, kp, row, n);
    });
    h->probe_rows++;
    CK(cudaGetLastError());
    return LBM_OK;
}

int lbm_advance(lbm_h h, int64_t n)
{
    if (!h) return LBM_ERR_ARG;
    if (n < 0) return fail(h, LBM_ERR_ARG, "negative step count");
    if (h->batch) return fail(h, LBM_ERR_ARG, "this hierarchy belongs to a batch: advance the batch");
    NvtxRange range("lbm_advance");
    if (!h->members.empty()) return batch_advance(h, n);
    for (int64_t s = 0; s < n; s++) {
        NvtxRange step("coarse step");
        const long long k = h->ncoarse;
        int rc;
        if (h->d.use_graphs && !h->timing && k >= 1) rc = run_graph(h, k);
        else rc = issue_coarse_step(h, k);
        if (rc != LBM_OK) return rc;
        h->ncoarse++;
        if (h->probes.n > 0 && h->probe_rows < h->probes.capacity) {
            rc = record_probes(h);
            if (rc != LBM_OK) return rc;
        }
    }
    return LBM_OK;
}

static int get_common(lbm_h h, int level, double *rho, double *u, double *pops, int on_device)
{
    const Level &v = h->lev[level];
    if (on_device) {
        dispatch(h, [&](auto s) { decltype(s)::macros(h, level, rho, u, pops); });
        CK(cudaGetLastError());
        return LBM_OK;
    }
    const size_t nr = rho ? v.N : 0, nu = u ? (size_t)h->D * v.N : 0, np = pops ? (size_t)h->Q * v.N : 0;
    double *tmp = (double *)tmp_alloc(h, (nr + nu + np + 1) * sizeof(double));
    if (!tmp) return fail(h, LBM_ERR_OOM, "staging buffer");
    double *dr = rho ? tmp : nullptr, *dd = u ? tmp + nr : nullptr, *dp = pops ? tmp + nr + nu : nullptr;
    dispatch(h, [&](auto s) { decltype(s)::macros(h, level, dr, dd, dp); });
    CK(cudaGetLastError());
    if (rho) CK(cudaMemcpyAsync(rho, dr, nr * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    if (u) CK(cudaMemcpyAsync(u, dd, nu * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    if (pops) CK(cudaMemcpyAsync(pops, dp, np * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    tmp_free(h, tmp);
    return LBM_OK;
}

int lbm_get_macros(lbm_h h, int level, double *rho_out, double *u_out, int on_device)
{
    if (!check_level(h, level)) return LBM_ERR_ARG;
    if (!rho_out && !u_out) return fail(h, LBM_ERR_ARG, "no output");
    return get_common(h, level, rho_out, u_out, nullptr, on_device);
}

int lbm_get_pops(lbm_h h, int level, double *f_out, int on_device)
{
    if (!check_level(h, level)) return LBM_ERR_ARG;
    if (!f_out) return fail(h, LBM_ERR_ARG, "f_out is NULL");
    return get_common(h, level, nullptr, nullptr, f_out, on_device);
}

int lbm_reduce(lbm_h h, int level, double out[4])
{
    if (!check_level(h, level)) return LBM_ERR_ARG;
    if (!out) return fail(h, LBM_ERR_ARG, "out is NULL");
    dispatch(h, [&](auto s) { decltype(s)::reduce(h, level); });
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(out, h->d_red, 4 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    int st = 0;
    CK(cudaMemcpy(&st, h->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (st & ST_NAN) return fail(h, LBM_ERR_DIVERGED, "NaN or Inf in level %d", level);
    return LBM_OK;
}

int lbm_reduce_async(lbm_h h, int level, double *out, int on_device)
{
    if (!check_level(h, level)) return LBM_ERR_ARG;
    if (!out) return fail(h, LBM_ERR_ARG, "out is NULL");
    cudaPointerAttributes pa{};
    CK(cudaPointerGetAttributes(&pa, out));
    if (on_device) {
        int dev = 0;
        CK(cudaGetDevice(&dev));
        if ((pa.type != cudaMemoryTypeDevice && pa.type != cudaMemoryTypeManaged) || pa.device != dev)
            return fail(h, LBM_ERR_ARG, "out is not device memory of the current device");
    } else if (pa.type != cudaMemoryTypeHost) {
        return fail(h, LBM_ERR_ARG, "out must be page-locked host memory for an asynchronous read");
    }
    dispatch(h, [&](auto s) { decltype(s)::reduce(h, level); });
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(out, h->d_red, 4 * sizeof(double), on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                       h->stream));
    return LBM_OK;
}

int lbm_check_status(lbm_h h)
{
    if (!h) return LBM_ERR_ARG;
    CK(cudaStreamSynchronize(h->stream));
    int st = 0;
    CK(cudaMemcpy(&st, h->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    CK(cudaMemset(h->d_status, 0, sizeof(int)));
    if (st & ST_TIMEOUT) return fail(h, LBM_ERR_TIMEOUT, "a bounded device-side wait gave up");
    if (st & ST_NEWTON) return fail(h, LBM_ERR_NEWTON, "Newton did not converge at a TF node");
    if (st & ST_NAN) return fail(h, LBM_ERR_DIVERGED, "NaN or Inf met");
    return LBM_OK;
}

int lbm_max_newton_iters(lbm_h h)
{
    if (!h) return LBM_ERR_ARG;
    int v = 0;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return LBM_ERR_CUDA;
    if (cudaMemcpy(&v, h->d_maxit, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return LBM_ERR_CUDA;
    return v;
}

int lbm_timing_enable(lbm_h h, int enable)
{
    if (!h) return LBM_ERR_ARG;
    CK(cudaStreamSynchronize(h->stream));
    h->timing = enable != 0;
    h->ev_pairs.clear();
    for (int l = 0; l < LBM_MAX_LEVELS; l++) {
        h->timing_ms[l] = 0.0;
        h->timing_launches[l] = 0;
    }
    return LBM_OK;
}

int lbm_timing_read(lbm_h h, double *ms_out, int64_t *launches_out)
{
    if (!h) return LBM_ERR_ARG;
    CK(cudaStreamSynchronize(h->stream));
    for (auto &pr : h->ev_pairs) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, h->ev_pool[pr.second], h->ev_pool[pr.second + 1]));
        h->timing_ms[pr.first] += ms;
        h->timing_launches[pr.first]++;
    }
    h->ev_pairs.clear();
    for (int l = 0; l < h->nl; l++) {
        if (ms_out) ms_out[l] = h->timing_ms[l];
        if (launches_out) launches_out[l] = h->timing_launches[l];
    }
    return LBM_OK;
}

int64_t lbm_launch_count(lbm_h h) { return h ? h->launches : 0; }
int64_t lbm_device_bytes(lbm_h h) { return h ? h->device_bytes : 0; }

int lbm_synchronize(lbm_h h)
{
    if (!h) return LBM_ERR_ARG;
    CK(cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

const char *lbm_last_error(lbm_h h) { return h ? h->err.c_str() : g_create_error.c_str(); }

void lbm_destroy(lbm_h h)
{
    if (!h) return;
    if (h->batch) return;  // members are destroyed with their batch
    if (h->stream) cudaStreamSynchronize(h->stream);
    for (auto *m : h->members) {
        m->batch = nullptr;
        m->own_stream = false;
        lbm_destroy(m);
    }
    h->members.clear();
    for (auto &kv : h->graphs) cudaGraphExecDestroy(kv.second);
    for (auto e : h->ev_pool) cudaEventDestroy(e);
    for (auto &b : h->bufs) {
        if (h->d.free) h->d.free(b.p, h->d.alloc_ctx);
        else cudaFree(b.p);
    }
    if (h->side) {
        cudaStreamSynchronize(h->side);
        cudaStreamDestroy(h->side);
    }
    for (int l = 0; l < LBM_MAX_LEVELS; l++)
        if (h->side2[l]) {
            cudaStreamSynchronize(h->side2[l]);
            cudaStreamDestroy(h->side2[l]);
        }
    for (int l = 0; l < LBM_MAX_LEVELS; l++)
        for (cudaEvent_t e : {h->ev_fork[l], h->ev_join[l], h->ev_parent[l], h->ev_bulk[l]})
            if (e) cudaEventDestroy(e);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
}

}  // extern "C"

// ================================================================== allocation-free reduction
// The level reduction above keeps its per-block partial sums in a buffer the handle
// allocated at creation.  This variant keeps them in a fixed array of static device
// memory instead, so the call itself never allocates: every GPU that loads the library
// holds the array (LBM_STATIC_REDUCE_PARTIALS x 4 doubles + 4, about 128 KB) until the
// process exits.  Host code cannot use the array's name as a device address; its
// address is looked up once per device with cudaGetSymbolAddress.
namespace {
constexpr int kStaticPartials = LBM_STATIC_REDUCE_PARTIALS;
constexpr int kStaticNodesPerBlock = 256 * 8;
static __device__ __align__(256) double g_static_reduce[kStaticPartials * 4 + 4];
std::mutex g_static_mtx;
double *g_static_addr[256] = {nullptr};
}  // namespace

extern "C" int lbm_reduce_static(lbm_h h, int level, double out[4])
{
    if (!check_level(h, level)) return LBM_ERR_ARG;
    if (!out) return fail(h, LBM_ERR_ARG, "out is NULL");
    const Level &v = h->lev[level];
    const long long blocks = (v.N + kStaticNodesPerBlock - 1) / kStaticNodesPerBlock;
    if (blocks > kStaticPartials)
        return fail(h, LBM_ERR_ARG,
                    "level %d has %lld box nodes; the static-scratch reduction handles at most %lld "
                    "(use lbm_reduce)", level, v.N, (long long)kStaticPartials * kStaticNodesPerBlock);
    int dev = 0;
    CK(cudaGetDevice(&dev));
    // the scratch address below is the current device's copy of the array: a handle
    // of another device would get a pointer its kernels cannot use
    if (dev != h->device)
        return fail(h, LBM_ERR_ARG, "the handle lives on device %d but device %d is current", h->device, dev);
    if (dev < 0 || dev >= 256) return fail(h, LBM_ERR_ARG, "device ordinal %d out of range", dev);
    double *scratch;
    {
        std::lock_guard<std::mutex> lock(g_static_mtx);
        if (!g_static_addr[dev]) {
            void *p = nullptr;
            CK(cudaGetSymbolAddress(&p, g_static_reduce));
            g_static_addr[dev] = (double *)p;
        }
        scratch = g_static_addr[dev];
    }
    double *result = scratch + (size_t)kStaticPartials * 4;
    const long long k = h->ncoarse << level;
    LevelDev dv = level_dev(h, level);
    // every block overwrites its own partial and the final kernel overwrites the
    // result, so nothing in the shared array has to be cleared between calls
    if (h->Q == 9) {
        if (h->d.storage == LBM_F64)
            k_reduce_partial<9, double><<<(int)blocks, 256, 0, h->stream>>>(dv.g, v.d_tag, (const double *)v.f[k & 1],
                                                                           v.d_wnode, scratch, h->d_status);
        else if (h->d.storage == LBM_F32)
            k_reduce_partial<9, float><<<(int)blocks, 256, 0, h->stream>>>(dv.g, v.d_tag, (const float *)v.f[k & 1],
                                                                          v.d_wnode, scratch, h->d_status);
        else
            k_reduce_partial<9, __half><<<(int)blocks, 256, 0, h->stream>>>(dv.g, v.d_tag, (const __half *)v.f[k & 1],
                                                                           v.d_wnode, scratch, h->d_status);
    } else {
        if (h->d.storage == LBM_F64)
            k_reduce_partial<19, double><<<(int)blocks, 256, 0, h->stream>>>(dv.g, v.d_tag, (const double *)v.f[k & 1],
                                                                            v.d_wnode, scratch, h->d_status);
        else if (h->d.storage == LBM_F32)
            k_reduce_partial<19, float><<<(int)blocks, 256, 0, h->stream>>>(dv.g, v.d_tag, (const float *)v.f[k & 1],
                                                                           v.d_wnode, scratch, h->d_status);
        else
            k_reduce_partial<19, __half><<<(int)blocks, 256, 0, h->stream>>>(
                dv.g, v.d_tag, (const __half *)v.f[k & 1], v.d_wnode, scratch, h->d_status);
    }
    k_reduce_final<<<1, 256, 0, h->stream>>>(scratch, (int)blocks, result);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(out, result, 4 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    int st = 0;
    CK(cudaMemcpy(&st, h->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (st & ST_NAN) return fail(h, LBM_ERR_DIVERGED, "NaN or Inf in level %d", level);
    return LBM_OK;
}


// ================================================================== batches
namespace {
constexpr int kBatchThreads = T2X * T2YT;                        // 256
constexpr int kBatchSeg = kBatchThreads / 16;                     // D2Q9 16-lane segments per work item

void emit_phases(std::vector<BatchPhase> &v, int l, int sub, int L)
{
    if (L > 1 || l > 0) v.push_back({PH_RH, l, sub, 0});
    if (l + 1 < L) {
        emit_phases(v, l + 1, 2 * sub, L);
        emit_phases(v, l + 1, 2 * sub + 1, L);
        v.back().join_next = 1;  // the child's last bulk pass is independent of what follows
    }
    if (l > 0) v.push_back({PH_GI, l, sub, 0});
    v.push_back({PH_BULK, l, sub, 0});
}

int build_batch(lbm_h b)
{
    const int n = (int)b->members.size(), L = b->nl;
    std::vector<LevelDev> lev((size_t)n * L);
    std::vector<IfaceDev> ifc((size_t)n * L);
    std::vector<int> pre_bulk((size_t)L * (n + 1), 0), pre_rh((size_t)L * (n + 1), 0), pre_gi((size_t)L * (n + 1), 0);
    std::vector<int> nb_recon((size_t)L * n, 0), nb_grad((size_t)L * n, 0), node_rh((size_t)L * n, 0),
        node_gi((size_t)L * n, 0);
    for (int hh = 0; hh < n; hh++) {
        lbm_h m = b->members[hh];
        for (int l = 0; l < L; l++) {
            lev[(size_t)hh * L + l] = level_dev(m, l);
            if (l > 0) ifc[(size_t)hh * L + l] = m->ifc[l].dev;
            const Level &v = m->lev[l];
            const int tiles = v.tiles[0] * v.tiles[1];
            // one node per thread for every member: a batch phase covers the interfaces
            // of all members together, so it has the throughput of a large interface
            const int cr = l > 0 ? m->ifc[l].dev.nTF : 0;
            const int ch = l + 1 < L ? m->ifc[l + 1].dev.nTF + m->ifc[l + 1].dev.nRing : 0;
            const int cg = l > 0 ? m->ifc[l].dev.nTF : 0, ci = l > 0 ? m->ifc[l].dev.nIE : 0;
            const bool nrh = true, ngi = true;
            const int pr = nrh ? kBatchThreads : kBatchSeg, pg = ngi ? kBatchThreads : kBatchSeg;
            const int nr = (cr + pr - 1) / pr, nh = (ch + pr - 1) / pr;
            const int ng = (cg + pg - 1) / pg, ni = (ci + pg - 1) / pg;
            nb_recon[(size_t)l * n + hh] = nr;
            nb_grad[(size_t)l * n + hh] = ng;
            node_rh[(size_t)l * n + hh] = nrh;
            node_gi[(size_t)l * n + hh] = ngi;
            const size_t o = (size_t)l * (n + 1);
            pre_bulk[o + hh + 1] = pre_bulk[o + hh] + tiles;
            pre_rh[o + hh + 1] = pre_rh[o + hh] + nr + nh;
            pre_gi[o + hh + 1] = pre_gi[o + hh] + ng + ni;
        }
    }
    lbm_h h = b;
    bool ok = true;
    BatchDev &B = b->bdev;
    B.n = n;
    B.L = L;
    B.lev = upload(b, lev, &ok);
    B.ifc = upload(b, ifc, &ok);
    B.pre_bulk = upload(b, pre_bulk, &ok);
    B.pre_rh = upload(b, pre_rh, &ok);
    B.nb_recon = upload(b, nb_recon, &ok);
    B.pre_gi = upload(b, pre_gi, &ok);
    B.nb_grad = upload(b, nb_grad, &ok);
    B.node_rh = upload(b, node_rh, &ok);
    B.node_gi = upload(b, node_gi, &ok);
    std::vector<BatchPhase> ph;
    emit_phases(ph, 0, 0, L);
    b->d_phases = upload(b, ph, &ok);
    b->nphases = (int)ph.size();
    b->phases = ph;
    b->work_bulk.assign(L, 0);
    b->work_rh.assign(L, 0);
    b->work_gi.assign(L, 0);
    for (int l = 0; l < L; l++) {
        b->work_bulk[l] = pre_bulk[(size_t)l * (n + 1) + n];
        b->work_rh[l] = pre_rh[(size_t)l * (n + 1) + n];
        b->work_gi[l] = pre_gi[(size_t)l * (n + 1) + n];
    }
    unsigned int *bar = (unsigned int *)dev_alloc(b, 4 * sizeof(unsigned int));
    b->d_status = (int *)dev_alloc(b, 2 * sizeof(int));
    if (!ok || !bar || !b->d_status) return fail(b, LBM_ERR_OOM, "batch tables");
    CK(cudaMemset(bar, 0, 4 * sizeof(unsigned int)));
    CK(cudaMemset(b->d_status, 0, 2 * sizeof(int)));
    b->d_maxit = b->d_status + 1;
    B.bar_count = bar;
    B.bar_gen = bar + 1;
    B.status = b->d_status;
    B.max_iters = b->d_maxit;
    B.barrier_ns = 2000000000ull;  // 2 s
    return LBM_OK;
}

template <typename S>
int batch_launch(lbm_h b, long long k0, int nsteps)
{
    lbm_h h = b;
    auto kern = k_batch<9, S, T2X, T2YT, T2NR>;
    if (b->batch_grid == 0) {
        int dev = 0, sms = 0, per_sm = 0;
        CK(cudaGetDevice(&dev));
        CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBatchThreads, 0));
        if (per_sm < 1) return fail(b, LBM_ERR_CUDA, "the batch kernel does not fit on an SM");
        b->batch_grid = sms * per_sm;
    }
    BatchDev B = b->bdev;
    const BatchPhase *ph = b->d_phases;
    int np = b->nphases;
    // a barrier that gave up in an earlier launch leaves its counter behind
    CK(cudaMemsetAsync(B.bar_count, 0, sizeof(unsigned int), b->stream));
    void *args[] = {&B, &ph, &np, &k0, &nsteps};
    CK(cudaLaunchCooperativeKernel((void *)kern, dim3(b->batch_grid), dim3(kBatchThreads), args, 0, b->stream));
    return LBM_OK;
}
}  // namespace

// The phase-launch structure: one launch per phase of the sub-cycle schedule, one CTA
// per work item of all members (k_batch_bulk / k_batch_rh / k_batch_gi).
template <typename S>
int batch_launch_phases(lbm_h b, long long k0, int nsteps)
{
    lbm_h h = b;
    const BatchDev B = b->bdev;
    for (int st = 0; st < nsteps; st++) {
        const long long k = k0 + st;
        for (const BatchPhase &ph : b->phases) {
            const int l = ph.level;
            const long long kl = (k << l) + ph.sub;
            if (ph.kind == PH_BULK) {
                if (b->work_bulk[l] > 0)
                    launch_chained(k_batch_bulk<9, S, T2X, T2YT, T2NR>, dim3(b->work_bulk[l]), dim3(kBatchThreads), 0,
                                   b->stream, B, l, kl);
            } else if (ph.kind == PH_RH) {
                const TimeW tw = l > 0 ? time_weights((int)(kl & 1), kl >> 1) : TimeW{};
                if (b->work_rh[l] > 0)
                    launch_chained(k_batch_rh<9, S>, dim3(b->work_rh[l]), dim3(kBatchThreads), 0, b->stream, B, l, kl, tw);
            } else {
                const TimeW tw = time_weights((int)(kl & 1), kl >> 1);
                if (b->work_gi[l] > 0)
                    launch_chained(k_batch_gi<9, S>, dim3(b->work_gi[l]), dim3(kBatchThreads), 0, b->stream, B, l, kl, tw);
            }
            b->launches++;
        }
    }
    CK(cudaGetLastError());
    return LBM_OK;
}

static int batch_advance(lbm_h b, int64_t n)
{
    lbm_h h = b;
    // every member counts the coarse steps done since its own initialisation
    long long k = b->members[0]->ncoarse;
    for (auto *m : b->members)
        if (m->ncoarse != k) return fail(b, LBM_ERR_ARG, "batch members were initialised at different steps");
    for (int64_t done = 0; done < n;) {
        const int chunk = (int)std::min<int64_t>(n - done, 1 << 20);
        int rc;
        if (b->batch_path == LBM_BATCH_PHASES) {
            if (b->d.storage == LBM_F64) rc = batch_launch_phases<double>(b, k + done, chunk);
            else if (b->d.storage == LBM_F32) rc = batch_launch_phases<float>(b, k + done, chunk);
            else rc = batch_launch_phases<__half>(b, k + done, chunk);
        } else {
            if (b->d.storage == LBM_F64) rc = batch_launch<double>(b, k + done, chunk);
            else if (b->d.storage == LBM_F32) rc = batch_launch<float>(b, k + done, chunk);
            else rc = batch_launch<__half>(b, k + done, chunk);
            b->launches++;
        }
        if (rc != LBM_OK) return rc;
        done += chunk;
    }
    for (auto *m : b->members) m->ncoarse += n;
    b->ncoarse = k + n;
    CK(cudaGetLastError());
    return LBM_OK;
}

extern "C" {

int lbm_create_batch(const lbm_hierarchy_desc *descs, int n, void *cuda_stream, lbm_h *out)
{
    if (!out) return fail(nullptr, LBM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!descs || n < 1) return fail(nullptr, LBM_ERR_ARG, "need at least one description");
    for (int i = 0; i < n; i++) {
        if (descs[i].lattice != 9) return fail(nullptr, LBM_ERR_BAD_DESC, "batches hold D2Q9 hierarchies");
        if (descs[i].storage != descs[0].storage || descs[i].n_levels != descs[0].n_levels)
            return fail(nullptr, LBM_ERR_BAD_DESC, "batch members need the same storage and level count");
    }
    lbm_h b = new lbm_hierarchy();
    b->d = descs[0];
    b->Q = 9;
    b->D = 2;
    b->nl = descs[0].n_levels;
    if (cudaGetDevice(&b->device) != cudaSuccess) {
        delete b;
        return fail(nullptr, LBM_ERR_CUDA, "cudaGetDevice failed");
    }
    if (cuda_stream) {
        b->stream = (cudaStream_t)cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete b;
            return fail(nullptr, LBM_ERR_CUDA, "cudaStreamCreateWithFlags failed");
        }
        b->own_stream = true;
    }
    for (int i = 0; i < n; i++) {
        lbm_h m = nullptr;
        const int rc = lbm_create_hierarchy(&descs[i], (void *)b->stream, &m);
        if (rc != LBM_OK) {
            const std::string e = std::string("member ") + std::to_string(i) + ": " + lbm_create_error();
            lbm_destroy(b);
            return fail(nullptr, rc, "%s", e.c_str());
        }
        m->batch = b;
        b->members.push_back(m);
    }
    const int rc = build_batch(b);
    if (rc != LBM_OK) {
        g_create_error = b->err;
        lbm_destroy(b);
        return rc;
    }
    *out = b;
    return LBM_OK;
}

int lbm_batch_member(lbm_h b, int i, lbm_h *member)
{
    if (!b || !member) return LBM_ERR_ARG;
    if (i < 0 || i >= (int)b->members.size())
        return fail(b, LBM_ERR_ARG, "member %d out of range [0,%d)", i, (int)b->members.size());
    *member = b->members[i];
    return LBM_OK;
}

int lbm_batch_check_barrier(lbm_h b, int skip_block, int64_t limit_us)
{
    lbm_h h = b;
    if (!b || b->members.empty()) return b ? fail(b, LBM_ERR_ARG, "not a batch") : LBM_ERR_ARG;
    if (limit_us < 1 || limit_us > 10000000) return fail(b, LBM_ERR_ARG, "limit must be in [1 us, 10 s]");
    int dev = 0, sms = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    CK(cudaMemsetAsync(b->bdev.bar_count, 0, 2 * sizeof(unsigned int), b->stream));
    CK(cudaMemsetAsync(b->d_status, 0, sizeof(int), b->stream));
    unsigned int *cnt = b->bdev.bar_count, *gen = b->bdev.bar_gen;
    int *st = b->d_status;
    unsigned long long lim = (unsigned long long)limit_us * 1000ull;
    void *args[] = {&cnt, &gen, &st, &lim, &skip_block};
    CK(cudaLaunchCooperativeKernel((void *)k_barrier_check, dim3(sms), dim3(32), args, 0, b->stream));
    CK(cudaStreamSynchronize(b->stream));
    int status = 0;
    CK(cudaMemcpy(&status, b->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    CK(cudaMemset(b->d_status, 0, sizeof(int)));
    CK(cudaMemset(b->bdev.bar_count, 0, 2 * sizeof(unsigned int)));
    if (status & ST_TIMEOUT) return fail(b, LBM_ERR_TIMEOUT, "a grid barrier wait gave up after %lld us", (long long)limit_us);
    return LBM_OK;
}

}  // extern "C"


// ================================================================== probes and state
extern "C" {

int lbm_set_probes(lbm_h h, int n, const double *xyz, int64_t capacity)
{
    if (!h || h->batch || !h->members.empty()) return h ? fail(h, LBM_ERR_ARG, "probes belong to single hierarchies") : LBM_ERR_ARG;
    if (h->masked) return fail(h, LBM_ERR_ARG, "probes take box hierarchies (the finest level holding a point is found by boxes)");
    if (n < 0 || n > 65536 || (n > 0 && !xyz) || capacity < 0 || capacity > (1 << 26))
        return fail(h, LBM_ERR_ARG, "bad probe count, positions or capacity");
    if ((int64_t)n * capacity > ((int64_t)1 << 28)) return fail(h, LBM_ERR_ARG, "probe buffer above 2^28 samples");
    std::vector<int> level(n), node((size_t)n * 8, 0);
    std::vector<double> w((size_t)n * 8, 0.0);
    const int nc = h->D == 3 ? 8 : 4;
    for (int j = 0; j < n; j++) {
        int found = -1;
        for (int l = h->nl - 1; l >= 0 && found < 0; l--) {
            const Level &v = h->lev[l];
            const double sc = std::ldexp(1.0, l);
            int64_t base[3];
            double fr[3];
            bool ok = true;
            for (int a = 0; a < 3; a++) {
                if (a >= h->D) {
                    base[a] = 0;
                    fr[a] = 0.0;
                    continue;
                }
                const double q = xyz[3 * j + a] * sc - (double)v.off[a];
                double fl = std::floor(q);
                fr[a] = q - fl;
                base[a] = (int64_t)fl;
                if (v.per[a]) continue;
                if (base[a] < 0 || base[a] + 1 > v.n[a] - 1) ok = false;
            }
            if (!ok) continue;
            int idx[8];
            double ww[8];
            for (int c = 0; c < nc && ok; c++) {
                int64_t p[3];
                double wc = 1.0;
                for (int a = 0; a < 3; a++) {
                    const int bit = (c >> a) & 1;
                    p[a] = base[a] + (a < h->D ? bit : 0) + v.off[a];
                    if (a < h->D) wc *= bit ? fr[a] : 1.0 - fr[a];
                }
                const long long id = node_of(h, l, p);
                if (id < 0) ok = false;
                else {
                    idx[c] = (int)(id % v.n[0] + v.px * (id / v.n[0]));  // slot of the node
                    ww[c] = wc;
                }
            }
            if (!ok) continue;
            found = l;
            for (int c = 0; c < nc; c++) {
                node[(size_t)j * 8 + c] = idx[c];
                w[(size_t)j * 8 + c] = ww[c];
            }
        }
        if (found < 0) return fail(h, LBM_ERR_ARG, "probe %d lies on no level's active cells", j);
        level[j] = found;
    }
    bool ok = true;
    ProbeDev P{};
    P.n = n;
    P.capacity = (int)capacity;
    P.level = upload(h, level, &ok);
    P.node = upload(h, node, &ok);
    P.w = upload(h, w, &ok);
    P.samples = (double *)dev_alloc(h, std::max<size_t>(1, (size_t)n * capacity) * sizeof(double));
    if (!h->d_levs) {
        std::vector<LevelDev> lv(h->nl);
        for (int l = 0; l < h->nl; l++) lv[l] = level_dev(h, l);
        h->d_levs = upload(h, lv, &ok);
        h->d_kstep = (long long *)dev_alloc(h, 64 * LBM_MAX_LEVELS * sizeof(long long));
    }
    if (!ok || !P.samples || !h->d_kstep) return fail(h, LBM_ERR_OOM, "probe buffers");
    h->probes = P;
    h->probe_rows = 0;
    return LBM_OK;
}

int lbm_get_probes(lbm_h h, double *out, int64_t *n_samples)
{
    if (!h || !n_samples) return h ? fail(h, LBM_ERR_ARG, "n_samples is NULL") : LBM_ERR_ARG;
    CK(cudaStreamSynchronize(h->stream));
    *n_samples = h->probe_rows;
    if (out && h->probes.n > 0 && h->probe_rows > 0)
        CK(cudaMemcpy(out, h->probes.samples, (size_t)h->probe_rows * h->probes.n * sizeof(double),
                      cudaMemcpyDeviceToHost));
    return LBM_OK;
}

// state = magic, version, lattice, storage, levels, coarse step, per-level box sizes,
// then each level's current populations and each interface's history, raw.
static const uint64_t kStateMagic = 0x4c424d4443535431ull;  // "LBMDCST1"

static size_t state_bytes(const lbm_h h)
{
    size_t b = 8 * 8 + 8 * LBM_MAX_LEVELS;
    const size_t ss = store_size(h->d.storage), as = arith_size(h->d.storage);
    for (int l = 0; l < h->nl; l++) b += (size_t)h->Q * h->lev[l].pitch * ss;
    for (int l = 1; l < h->nl; l++)
        b += (size_t)3 * h->Q * std::max(1, h->ifc[l].dev.nTF) * as + (size_t)3 * 4 * std::max(1, h->ifc[l].dev.nRing) * as;
    return b;
}

// 64-bit FNV-1a of the FP16 storage shift and of the refinement masks, so that a state
// is loaded only where its stored populations mean the same values on the same nodes
static uint64_t shift_key(const lbm_h h)
{
    uint64_t k = 1469598103934665603ull;
    const unsigned char *b = (const unsigned char *)h->shift;
    for (size_t i = 0; i < sizeof(h->shift); i++) k = (k ^ b[i]) * 1099511628211ull;
    for (int l = 1; l < h->nl; l++)  // and the staircase regions: a state belongs to its geometry
        for (uint8_t m : h->mask[l]) k = (k ^ (uint64_t)(m != 0)) * 1099511628211ull;
    return k;
}

int lbm_save_state(lbm_h h, void *buf, size_t *len)
{
    if (!h || !len) return h ? fail(h, LBM_ERR_ARG, "len is NULL") : LBM_ERR_ARG;
    if (!h->members.empty()) return fail(h, LBM_ERR_ARG, "save the members of a batch one by one");
    const size_t need = state_bytes(h);
    if (!buf) {
        *len = need;
        return LBM_OK;
    }
    if (*len < need) return fail(h, LBM_ERR_ARG, "buffer of %zu bytes, %zu needed", *len, need);
    CK(cudaStreamSynchronize(h->stream));
    uint64_t *hd = (uint64_t *)buf;
    hd[0] = kStateMagic;
    hd[1] = 1;
    hd[2] = (uint64_t)h->Q;
    hd[3] = (uint64_t)h->d.storage;
    hd[4] = (uint64_t)h->nl;
    hd[5] = (uint64_t)h->ncoarse;
    hd[6] = shift_key(h);
    hd[7] = 0;
    for (int l = 0; l < LBM_MAX_LEVELS; l++) hd[8 + l] = l < h->nl ? (uint64_t)h->lev[l].N : 0;
    char *p = (char *)buf + 8 * 8 + 8 * LBM_MAX_LEVELS;
    const size_t ss = store_size(h->d.storage), as = arith_size(h->d.storage);
    for (int l = 0; l < h->nl; l++) {
        const Level &v = h->lev[l];
        const size_t b = (size_t)h->Q * v.pitch * ss;
        CK(cudaMemcpy(p, v.f[(h->ncoarse << l) & 1], b, cudaMemcpyDeviceToHost));
        p += b;
    }
    for (int l = 1; l < h->nl; l++) {
        const IfaceDev &I = h->ifc[l].dev;
        const size_t bf = (size_t)3 * h->Q * std::max(1, I.nTF) * as, bm = (size_t)3 * 4 * std::max(1, I.nRing) * as;
        CK(cudaMemcpy(p, I.hist_f, bf, cudaMemcpyDeviceToHost));
        p += bf;
        CK(cudaMemcpy(p, I.hist_m, bm, cudaMemcpyDeviceToHost));
        p += bm;
    }
    *len = need;
    return LBM_OK;
}

int lbm_load_state(lbm_h h, const void *buf, size_t len)
{
    if (!h || !buf) return h ? fail(h, LBM_ERR_ARG, "buf is NULL") : LBM_ERR_ARG;
    if (!h->members.empty()) return fail(h, LBM_ERR_ARG, "load the members of a batch one by one");
    const size_t need = state_bytes(h);
    const uint64_t *hd = (const uint64_t *)buf;
    if (len < need || hd[0] != kStateMagic || hd[1] != 1 || hd[2] != (uint64_t)h->Q ||
        hd[3] != (uint64_t)h->d.storage || hd[4] != (uint64_t)h->nl || hd[6] != shift_key(h))
        return fail(h, LBM_ERR_ARG, "state does not belong to this hierarchy (lattice, storage, shift, levels or size)");
    for (int l = 0; l < h->nl; l++)
        if (hd[8 + l] != (uint64_t)h->lev[l].N) return fail(h, LBM_ERR_ARG, "level %d has another box", l);
    CK(cudaStreamSynchronize(h->stream));
    h->ncoarse = (long long)hd[5];
    const char *p = (const char *)buf + 8 * 8 + 8 * LBM_MAX_LEVELS;
    const size_t ss = store_size(h->d.storage), as = arith_size(h->d.storage);
    for (int l = 0; l < h->nl; l++) {
        const Level &v = h->lev[l];
        const size_t b = (size_t)h->Q * v.pitch * ss;
        CK(cudaMemcpy(v.f[(h->ncoarse << l) & 1], p, b, cudaMemcpyHostToDevice));
        p += b;
    }
    for (int l = 1; l < h->nl; l++) {
        const IfaceDev &I = h->ifc[l].dev;
        const size_t bf = (size_t)3 * h->Q * std::max(1, I.nTF) * as, bm = (size_t)3 * 4 * std::max(1, I.nRing) * as;
        CK(cudaMemcpy(I.hist_f, p, bf, cudaMemcpyHostToDevice));
        p += bf;
        CK(cudaMemcpy(I.hist_m, p, bm, cudaMemcpyHostToDevice));
        p += bm;
    }
    return LBM_OK;
}

}  // extern "C"


// ================================================================== autotuner
extern "C" {

int lbm_set_tile_config(lbm_h h, int level, int cfg)
{
    if (!check_level(h, level)) return LBM_ERR_ARG;
    if (cfg < 0 || cfg >= LBM_TILE_CONFIGS) return fail(h, LBM_ERR_ARG, "tile configuration %d out of range", cfg);
    if (h->lev[level].tile_cfg != cfg) {
        for (auto &kv : h->graphs) cudaGraphExecDestroy(kv.second);  // graphs bake the launch shapes
        h->graphs.clear();
        h->graph_launches.clear();
    }
    h->lev[level].tile_cfg = cfg;
    return h->D == 3 ? plan_chunks(h, level) : LBM_OK;
}

int lbm_debug_withhold_copy(lbm_h h, int level, int bx, int by, int bz, int k, int64_t limit_us)
{
    if (!h) return LBM_ERR_ARG;
    if (h->batch || !h->members.empty()) return fail(h, LBM_ERR_ARG, "not for batches");
    if (level < 0) {
        h->withhold_level = h->withhold_block = h->withhold_k = -1;
    } else {
        if (!check_level(h, level)) return LBM_ERR_ARG;
        const Level &v = h->lev[level];
        if (h->Q != 19) return fail(h, LBM_ERR_ARG, "the staged bulk kernel is the D3Q19 one");
        if (bx < 0 || by < 0 || bz < 0 || bx >= v.tiles[0] || by >= v.tiles[1] || bz >= v.tiles[2] || k < 0 ||
            limit_us < 1 || limit_us > 10000000)
            return fail(h, LBM_ERR_ARG, "block, stage or limit out of range");
        h->withhold_level = level;
        h->withhold_block = bx + v.tiles[0] * (by + v.tiles[1] * bz);
        h->withhold_k = k;
        h->withhold_limit_ns = (unsigned long long)limit_us * 1000ull;
    }
    for (auto &kv : h->graphs) cudaGraphExecDestroy(kv.second);
    h->graphs.clear();
    h->graph_launches.clear();
    return LBM_OK;
}

int lbm_set_interface_mapping(lbm_h h, int mode)
{
    if (!h) return LBM_ERR_ARG;
    if (h->batch || !h->members.empty())
        return fail(h, LBM_ERR_ARG, "the interface mapping of a batch is fixed when it is created");
    if (mode != LBM_IFACE_AUTO && mode != LBM_IFACE_NODE && mode != LBM_IFACE_SEGMENT)
        return fail(h, LBM_ERR_ARG, "interface mapping %d is not AUTO, NODE or SEGMENT", mode);
    if (h->if_mode != mode) {
        for (auto &kv : h->graphs) cudaGraphExecDestroy(kv.second);  // graphs bake the launch shapes
        h->graphs.clear();
        h->graph_launches.clear();
    }
    h->if_mode = mode;
    return LBM_OK;
}

int lbm_get_tile_config(lbm_h h, int level, int *cfg)
{
    if (!check_level(h, level)) return LBM_ERR_ARG;
    if (!cfg) return fail(h, LBM_ERR_ARG, "cfg is NULL");
    *cfg = h->lev[level].tile_cfg;
    return LBM_OK;
}

int lbm_batch_set_path(lbm_h b, int path)
{
    if (!b || b->members.empty()) return b ? fail(b, LBM_ERR_ARG, "not a batch") : LBM_ERR_ARG;
    if (path != LBM_BATCH_PERSISTENT && path != LBM_BATCH_PHASES) return fail(b, LBM_ERR_ARG, "unknown launch structure %d", path);
    b->batch_path = path;
    return LBM_OK;
}

int lbm_batch_get_path(lbm_h b)
{
    if (!b || b->members.empty()) return b ? fail(b, LBM_ERR_ARG, "not a batch") : LBM_ERR_ARG;
    return b->batch_path;
}

// batches: the launch structure of a coarse step (one persistent launch, or one launch
// per phase), each timed over reps coarse steps of the live state, the faster kept
static int autotune_batch(lbm_h b, int reps, double *us_out)
{
    lbm_h h = b;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    double us[2] = {0.0, 0.0};
    const int paths[2] = {LBM_BATCH_PERSISTENT, LBM_BATCH_PHASES};
    for (int p = 0; p < 2; p++) {
        b->batch_path = paths[p];
        int rc = batch_advance(b, 1);  // warm-up
        if (rc != LBM_OK) return rc;
        CK(cudaEventRecord(e0, b->stream));
        rc = batch_advance(b, reps);
        if (rc != LBM_OK) return rc;
        CK(cudaEventRecord(e1, b->stream));
        CK(cudaEventSynchronize(e1));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        us[p] = 1e3 * ms / reps;
        if (us_out) us_out[p] = us[p];
    }
    b->batch_path = us[1] < us[0] ? LBM_BATCH_PHASES : LBM_BATCH_PERSISTENT;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    CK(cudaGetLastError());
    return LBM_OK;
}

int lbm_autotune(lbm_h h, int reps, double *us_out)
{
    if (!h || h->batch) return h ? fail(h, LBM_ERR_ARG, "autotune a hierarchy or a whole batch") : LBM_ERR_ARG;
    if (reps < 1 || reps > 10000) return fail(h, LBM_ERR_ARG, "reps must be in [1, 10000]");
    if (!h->members.empty()) return autotune_batch(h, reps, us_out);
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    for (int l = 0; l < h->nl; l++) {
        Level &v = h->lev[l];
        const long long k = h->ncoarse << l;
        const void *src = v.f[k & 1];
        void *dst = v.f[(k + 1) & 1];  // the state stays in src: timing does not advance it
        double best = 1e300;
        int best_c = 0;
        for (int c = 0; c < LBM_TILE_CONFIGS; c++) {
            const int saved = v.tile_cfg;
            v.tile_cfg = c;
            if (h->D == 3 && plan_chunks(h, l) != LBM_OK) return LBM_ERR_CUDA;
            dispatch(h, [&](auto s) { decltype(s)::bulk(h, l, src, dst); });  // warm-up
            CK(cudaEventRecord(e0, h->stream));
            for (int r = 0; r < reps; r++) dispatch(h, [&](auto s) { decltype(s)::bulk(h, l, src, dst); });
            CK(cudaEventRecord(e1, h->stream));
            CK(cudaEventSynchronize(e1));
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, e0, e1));
            v.tile_cfg = saved;
            if (h->D == 3 && plan_chunks(h, l) != LBM_OK) return LBM_ERR_CUDA;
            const double us = 1e3 * ms / reps;
            if (us_out) us_out[l * LBM_TILE_CONFIGS + c] = us;
            if (us < best) {
                best = us;
                best_c = c;
            }
        }
        const int rc = lbm_set_tile_config(h, l, best_c);
        if (rc != LBM_OK) return rc;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    CK(cudaGetLastError());
    return LBM_OK;
}

}  // extern "C"
