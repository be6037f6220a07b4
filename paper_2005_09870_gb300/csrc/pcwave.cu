// libpcwave: C-ABI entry points, host planner and launches (see include/pcwave.h).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <atomic>
#include <mutex>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/pcwave.h"
#include "pcw_geom.cuh"
#include "pcw_kernels.cuh"
#include "pcw_asm2d.cuh"
#include "pcw_bwd2d.cuh"
#include "pcw_taps.h"
#include "pcw_svir_gpu.cuh"
#include "pcw_alg1.cuh"

using namespace pcw;

namespace {

thread_local std::string g_noh_error = "no error";
std::atomic<long long> g_launches{0};
inline void count_launch(long long k = 1) { g_launches.fetch_add(k, std::memory_order_relaxed); }

struct BandPlan {
    int b, rows, jlo, jhi, k0;
    AsmCfg cfg;    // forward rows
    size_t smem;
    AsmCfg cfg_b;  // adjoint rows (same groups, their own arena)
    size_t smem_b;
};

}  // namespace

struct pc_op {
    pc_desc desc{};
    int Lf = 0, K = 0, Ku = 0, nb = 0;
    int64_t N = 0, nnz = 0;
    size_t esz = 4;  // bytes per element of the precision type
    double h[64]{};
    std::vector<int64_t> row_ptr_h;
    std::vector<BandPlan> plan;
    FiltDev fd{};
    int wofs[MAXL + 2]{};
    int wav_total = 0;
    int64_t Ftotal = 0, Gtotal = 0;
    int mwords = 1, ts0 = 1, ts1 = 1, tpa0 = 1, tpa1 = 1;
    // device buffers
    void* u_d = nullptr;
    void* v_d = nullptr;
    double* taps64_d = nullptr;
    double* wav64_d = nullptr;
    void* tapsT_d = nullptr;
    void* wavT_d = nullptr;
    void* F_d = nullptr;
    void* G_d = nullptr;
    void* dF_d = nullptr;  // backward scratch: dL/dF
    void* dG_d = nullptr;  // backward scratch: dL/dG
    void* S_d = nullptr;   // 2-D: stage-1 values s of every row (assembly), then dL/ds (backward)
    void* od_d = nullptr;   // device copy of the operator descriptor for k_s_tiles
    unsigned long long* amask_d = nullptr;  // backward scratch: active terms per row (2-D)
    int64_t Stotal = 0;
    int64_t FTtotal = 0;  // term-contiguous copy of F (FP32 backward), after dG in its scratch
    BwdDev bd{};
    int64_t* row_ptr_d = nullptr;
    void* theta_d = nullptr;
    __nv_bfloat16* theta16_d = nullptr;
    void* fista_d = nullptr;       // solver scratch: y, r, g (3 N elements), then two doubles
    unsigned long long* bdesc_d = nullptr;  // column-block descriptors for one-column products
    unsigned* boff_d = nullptr;             // offset of each described block within its row
    int bdesc_stride = 0;                   // slots per row (most kept blocks of any row band)
    void* thetaT_d = nullptr;               // transposed copy of the stored values (same pattern)
    long long theta_gen = 0, thetaT_gen = -1;  // assemblies so far / the one thetaT_d reflects
    unsigned* xsplit_d = nullptr;  // 16 right-hand sides split into packed BF16 hi / lo (tensor-core apply)
    unsigned long long* masks_d = nullptr;
    void* wl_d = nullptr;   // per-pixel window list (slots x N)
    int wl_slots = 0;       // slots allocated and in use
    int* cnt_d = nullptr;   // scratch int for the slot count
    int* dfoff_d = nullptr; // block offsets of the dL/dF launch per band
    int* err_d = nullptr;
    int64_t dev_bytes = 0;
    bool assembled = false;
    bool prepared = false;  // stage 0 ran for the current parameters
    // FP32 row assembly through the persistent work queue (one launch over all bands)
    BatchItem* q_items_d = nullptr;
    BatchItem* q_items_b_d = nullptr;  // the same items with the adjoint rows' plan
    OpDev<float>* q_op_d = nullptr;
    int* q_counter_d = nullptr;
    int q_nitems = 0, q_grid = 0, q_kind = 0;
    size_t q_smem = 0, q_smem_b = 0;
    std::string err = "no error";
};

// Work items of one kernel kind (see k_assemble_batch) in a contiguous range of the queue.
struct QGroup {
    int kind, start, count, grid;
};

struct pc_batch {
    std::vector<pc_op*> ops;
    std::vector<OpDev<float>> od;  // host copy of the operators' descriptors (refreshed per run)
    OpDev<float>* ops_d = nullptr;
    BatchItem* items_d = nullptr;
    int* counter_d = nullptr;  // one counter per group
    int nitems = 0;
    std::vector<QGroup> groups;
    size_t smem = 0;
    int kernels_per_run = 0;
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    // the kinds' persistent launches run side by side: group g > 0 on side[g - 1], forked
    // from and joined back into the run's stream by events
    std::vector<cudaStream_t> side;
    std::vector<cudaEvent_t> fork, join;
    // every operator's stage 0 and stage-1 sums run on one of these streams (round robin),
    // forked from the run's stream by prep_fork and joined back before the persistent launches
    std::vector<cudaStream_t> prep;
    std::vector<cudaEvent_t> prep_join;
    cudaEvent_t prep_fork = nullptr;
};

namespace {

pc_status fail(pc_op* h, pc_status st, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (h)
        h->err = buf;
    else
        g_noh_error = buf;
    return st;
}

#define PC_CUDA(h, call)                                                                               \
    do {                                                                                               \
        cudaError_t e_ = (call);                                                                       \
        if (e_ != cudaSuccess)                                                                         \
            return fail(h, e_ == cudaErrorMemoryAllocation ? PC_ERR_OOM : PC_ERR_CUDA, "%s: %s (%s:%d)", \
                        #call, cudaGetErrorString(e_), __FILE__, __LINE__);                            \
    } while (0)

bool is_pow2(int x) { return x > 0 && (x & (x - 1)) == 0; }

pc_status check_desc(const pc_desc* d, pc_op* h)
{
    if (!d) return fail(h, PC_ERR_INVALID_ARG, "desc is NULL");
    if (d->dim != 1 && d->dim != 2) return fail(h, PC_ERR_INVALID_ARG, "dim must be 1 or 2 (got %d)", d->dim);
    if (!is_pow2(d->n) || d->n < 2) return fail(h, PC_ERR_INVALID_ARG, "n must be a power of two >= 2 (got %d)", d->n);
    if (d->dim == 2 && d->n > 16384) return fail(h, PC_ERR_UNSUPPORTED, "2-D side > 16384");
    if (d->dim == 1 && d->n > (1 << 28)) return fail(h, PC_ERR_UNSUPPORTED, "1-D length > 2^28");
    if (d->levels < 1 || d->levels > MAXL || (d->n >> d->levels) < 1)
        return fail(h, PC_ERR_INVALID_ARG, "levels must satisfy 1 <= L <= %d and n >> L >= 1", MAXL);
    if (d->delta < 1 || d->delta > 10) return fail(h, PC_ERR_INVALID_ARG, "delta must be in 1..10");
    if (d->m < 1 || d->m > 64 * MAXW) return fail(h, PC_ERR_UNSUPPORTED, "m must be in 1..%d", 64 * MAXW);
    if (d->radius < 0 || d->radius > 64) return fail(h, PC_ERR_UNSUPPORTED, "radius must be in 0..64");
    if (d->gap < -1) return fail(h, PC_ERR_INVALID_ARG, "gap must be -1 (dense) or >= 0");
    if (d->order != 0 && d->order != 1) return fail(h, PC_ERR_INVALID_ARG, "order must be 0 or 1");
    if (d->precision != PC_FP32 && d->precision != PC_FP64) return fail(h, PC_ERR_INVALID_ARG, "bad precision");
    if (d->store_bf16 && d->precision != PC_FP32) return fail(h, PC_ERR_INVALID_ARG, "store_bf16 needs PC_FP32");
    if (d->family != PC_DAUBECHIES && d->family != PC_SYMMLET)
        return fail(h, PC_ERR_INVALID_ARG, "family must be PC_DAUBECHIES or PC_SYMMLET (got %d)", d->family);
    if (d->gap < 0) {
        int64_t N = (d->dim == 2) ? (int64_t)d->n * d->n : d->n;
        if (N > 16384) return fail(h, PC_ERR_UNSUPPORTED, "dense pattern limited to N <= 16384");
    }
    return PC_OK;
}

struct Geo {
    int d, n, L, Lf, r, gap, nb;
};

Geo geo_of(const pc_desc* d)
{
    Geo g;
    g.d = d->dim;
    g.n = d->n;
    g.L = d->levels;
    g.Lf = 2 * d->delta;
    g.r = d->radius;
    g.gap = d->gap;
    g.nb = num_bands(g.d, g.L);
    return g;
}

int64_t band_rows(const Geo& g, int b)
{
    Band B = band_info(g.d, g.n, g.L, b);
    return (g.d == 2) ? (int64_t)B.nj * B.nj : B.nj;
}

int64_t row_length(const Geo& g, int b, int l0, int l1)
{
    int64_t acc = 0;
    for (int b2 = 0; b2 < g.nb; ++b2)
        if (block_kept(g.d, g.n, g.L, g.gap, b, b2)) acc += block_count(g.d, g.n, g.L, g.Lf, g.r, g.gap, b, l0, l1, b2);
    return acc;
}

// decode a canonical index into band / translates
void decode(const Geo& g, int64_t s, int* b, int* l0, int* l1)
{
    for (int bb = g.nb - 1; bb >= 0; --bb) {
        Band B = band_info(g.d, g.n, g.L, bb);
        int64_t sz = band_rows(g, bb);
        if (s >= B.off && s < B.off + sz) {
            *b = bb;
            int rl = (int)(s - B.off);
            *l0 = (g.d == 2) ? rl / B.nj : 0;
            *l1 = (g.d == 2) ? rl % B.nj : rl;
            return;
        }
    }
    *b = -1;
}

pc_status plan_nnz(const Geo& g, std::vector<int64_t>* row_ptr, int64_t* nnz)
{
    int64_t N = (g.d == 2) ? (int64_t)g.n * g.n : g.n;
    if (row_ptr) row_ptr->assign(N + 1, 0);
    int64_t acc = 0;
    for (int b = 0; b < g.nb; ++b) {
        Band B = band_info(g.d, g.n, g.L, b);
        int nj = B.nj;
        // a row's length depends on its translate only through l mod 2^(j2 - j) <= 2^gap
        // (stencils toward finer column bands): cache per phase
        const int P = 1 << std::min(std::max(g.gap, 0), 12);
        const int p0n = std::min(nj, P), p1n = std::min(nj, P);
        std::vector<int64_t> cache((size_t)((g.d == 2) ? p0n : 1) * p1n, -1);
        for (int l0 = 0; l0 < ((g.d == 2) ? nj : 1); ++l0)
            for (int l1 = 0; l1 < nj; ++l1) {
                int64_t len;
                size_t ci = (size_t)((g.d == 2) ? (l0 % p0n) : 0) * p1n + (l1 % p1n);
                if (cache[ci] < 0) cache[ci] = row_length(g, b, l0, l1);
                len = cache[ci];
                if (row_ptr) (*row_ptr)[B.off + (int64_t)l0 * ((g.d == 2) ? nj : 0) + l1] = acc;
                acc += len;
            }
    }
    if (row_ptr) (*row_ptr)[N] = acc;
    *nnz = acc;
    return PC_OK;
}

// Persistent queue kernels, one instantiation per kind: 1 = 1-D rows, else the 2-D filter
// template length.
int item_kind(int dim, int lft) { return dim == 1 ? 1 : lft; }

using QueueKernel = decltype(&k_assemble_batch<8>);
QueueKernel queue_kernel(int kind)
{
    switch (kind) {
    case 1: return k_assemble_batch<1>;
    case 2: return k_assemble_batch<2>;
    case 4: return k_assemble_batch<4>;
    case 8: return k_assemble_batch<8>;
    default: return k_assemble_batch<20>;
    }
}

using BwdQueueKernel = decltype(&k_backward_queue<8>);
BwdQueueKernel bwd_queue_kernel(int lft)
{
    switch (lft) {
    case 2: return k_backward_queue<2>;
    case 4: return k_backward_queue<4>;
    case 8: return k_backward_queue<8>;
    default: return k_backward_queue<20>;
    }
}

// Resident CTAs of a 256-thread kernel over the device (the grid of a persistent launch).
template <typename K>
int persistent_grid(K fn, size_t smem)
{
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 256, smem);
    return std::max(1, sms * std::max(1, per_sm));
}

// per-axis maxima of the ranges a row group meets, over the translate phases of a band
struct AxisMax {
    int A;              // region count
    int c;              // stage-1 output count
    int lev[MAXL + 2];  // cascade counts per level
};

AxisMax axis_max(const Geo& g, int j, int e, int nj, int k0, int jhi)
{
    AxisMax M{};
    const int lim = std::min(nj, 1 << std::min(12, std::max(1, jhi - j + 2)));
    for (int l = 0; l < lim; ++l) {
        Range A = region0(j, e, l, g.r, g.Lf, g.n);
        M.A = std::max(M.A, A.cnt);
        Range c;
        int lvl;
        if (k0 == 0) {
            c = range_cascade(A, g.Lf, g.n >> 1);
            lvl = 1;
        } else {
            c = range_filter(A, 1 << k0, 0, wav_len(k0, g.Lf), g.n >> k0);
            lvl = k0;
        }
        M.c = std::max(M.c, c.cnt);
        M.lev[lvl] = std::max(M.lev[lvl], c.cnt);
        Range p = c;
        for (int jj = lvl + 1; jj <= jhi; ++jj) {
            p = range_cascade(p, g.Lf, g.n >> jj);
            M.lev[jj] = std::max(M.lev[jj], p.cnt);
        }
    }
    return M;
}

int64_t round_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

// filter-length template of the 2-D kernels (shorter filters run zero-padded)
int lf_template(int Lf) { return Lf <= 2 ? 2 : Lf <= 4 ? 4 : Lf <= 8 ? 8 : 20; }

// Checks, for every translate phase of band b, that each kept stencil window lies inside the
// coefficient range the row's localized transform computes at that level (the kernels copy
// windows without bounds checks when the range does not wrap).
bool stencils_inside(const Geo& g, int b, int k0, int jhi)
{
    Band B = band_info(g.d, g.n, g.L, b);
    const int lim = std::min(B.nj, 1 << std::min(12, std::max(1, jhi - B.j + 2)));
    for (int axis = (g.d == 2 ? 0 : 1); axis < 2; ++axis) {
        const int e = axis == 0 ? B.e0 : B.e1;
        for (int l = 0; l < lim; ++l) {
            Range rng[MAXL + 2];
            Range A = region0(B.j, e, l, g.r, g.Lf, g.n);
            int lvl0;
            if (k0 == 0) {
                rng[1] = range_cascade(A, g.Lf, g.n >> 1);
                lvl0 = 1;
            } else {
                rng[k0] = range_filter(A, 1 << k0, 0, wav_len(k0, g.Lf), g.n >> k0);
                lvl0 = k0;
            }
            for (int jj = lvl0 + 1; jj <= jhi; ++jj) rng[jj] = range_cascade(rng[jj - 1], g.Lf, g.n >> jj);
            for (int b2 = 0; b2 < g.nb; ++b2) {
                if (!block_kept(g.d, g.n, g.L, g.gap, b, b2)) continue;
                Band B2 = band_info(g.d, g.n, g.L, b2);
                if (B2.j < lvl0 || (k0 > 0 && B2.j == k0)) return false;  // level not produced
                const int e2 = axis == 0 ? B2.e0 : B2.e1;
                int f, W;
                stencil(B.j, e, l, B2.j, e2, g.r, g.Lf, g.n, g.gap < 0, &f, &W);
                const Range& R = rng[B2.j];
                if (!R.full && g.gap >= 0 && (f < R.lo || f + W > R.lo + R.cnt)) return false;
            }
        }
    }
    return true;
}

// Plan of one row band: thread-group size gt (0 = heuristic from the region area), groups per
// CTA, stage-1 batch of s rows, per-group arena (the maximum over translate phases of what
// every stage holds at once) and the dynamic shared memory of a CTA.
pc_status plan_band(pc_op* h, const Geo& g, int b, int gt_req, BandPlan* out)
{
    const size_t es = h->esz;
    Band B = band_info(g.d, g.n, g.L, b);
    BandPlan bp{};
    bp.b = b;
    bp.rows = (int)band_rows(g, b);
    const int dense = g.gap < 0;
    bp.jlo = dense ? 1 : std::max(1, B.j - g.gap);
    bp.jhi = dense ? g.L : std::min(g.L, B.j + g.gap);
    bp.k0 = (g.d == 2) ? bp.jlo - 1 : 0;
    int64_t need = 0, bneed = -1;  // forward / adjoint arena (bneed < 0: the same)
    int gt, batch = 1;
    AxisMax M1 = axis_max(g, B.j, B.e1, B.nj, bp.k0, bp.jhi);
    if (g.d == 1) {
        // X then alternating (a|d) outputs at the two arena ends
        int64_t prev = M1.A;
        for (int jj = 1; jj <= bp.jhi; ++jj) {
            int64_t cur = 2 * (int64_t)M1.lev[jj];
            need = std::max(need, prev + cur);
            prev = cur;
        }
        gt = gt_req ? gt_req : ((M1.A > 256) ? 64 : 32);
    } else {
        AxisMax M0 = axis_max(g, B.j, B.e0, B.nj, bp.k0, bp.jhi);
        const int64_t area = (int64_t)M0.A * M1.A;
        gt = gt_req ? gt_req : (area <= 768 ? 32 : area <= 2048 ? 64 : area <= 6144 ? 128 : 256);
        const int lo1 = bp.k0 > 0;
        // forward row (asm2d_row): padded line arrays; every size below is monotone in the
        // counts, so the per-axis maxima bound every translate phase
        const int mg = pass_margin(g.Lf, lf_template(g.Lf));
        const int64_t XP = lo1 ? (M1.A | 1) : odd_pitch(M1.A, mg);  // s rows (padded unless the first pass is phi_k0)
        const int lvl0 = lo1 ? bp.k0 : 1;
        const int64_t Yf = lo1 ? (int64_t)M0.A * M1.c : 2 * (int64_t)padded_size(M1.c, M0.A, mg);
        const int64_t Zf = padded_size(M0.c, M1.c, mg) + (lo1 ? 0 : 3 * (int64_t)M0.c * M1.c);
        // s rows per stage-1 step: the whole region when it fits a ~96 KB-per-CTA budget,
        // else as many rows as the budget allows (at least 8 pixels per thread)
        const int64_t budget = (96 * 1024 / (int64_t)es) / std::max(1, 256 / gt);
        const int64_t room = std::max<int64_t>(budget - Yf, (int64_t)8 * gt);
        batch = (int)std::max<int64_t>(1, std::min<int64_t>(M0.A, room / XP));
        need = std::max<int64_t>((lo1 ? (int64_t)batch * XP : padded_size(batch, M1.A, mg)) + Yf, Zf + Yf);
        int64_t prevZ = Zf;
        for (int jj = lvl0 + 1; jj <= bp.jhi; ++jj) {
            const int64_t ysz = 2 * (int64_t)padded_size(M1.lev[jj], M0.lev[jj - 1], mg);
            const int64_t zsz = padded_size(M0.lev[jj], M1.lev[jj], mg) + 3 * (int64_t)M0.lev[jj] * M1.lev[jj];
            need = std::max(need, std::max(prevZ + ysz, zsz + ysz));
            prevZ = zsz;
        }
        // adjoint row (bwd2d_row, and the atomic adjoint k_backward): compact arrays
        // (bwd2d_row keeps ADJ_SLACK elements below the arena end and ADJ_SLACK rows after Z)
        // (axis-1 ranges one longer: bwd2d_row pads them to odd counts)
        const int64_t c1 = M1.c + 1;
        const int64_t Yb = (int64_t)(lo1 ? 1 : 2) * M0.A * c1 + ADJ_SLACK;
        const int64_t Zb = (int64_t)(lo1 ? 1 : 4) * M0.c * c1;
        bneed = std::max<int64_t>((int64_t)batch * M1.A + Yb, std::max(Zb + Yb, Zb + ADJ_SLACK * c1));
        prevZ = Zb;
        for (int jj = lvl0 + 1; jj <= bp.jhi; ++jj) {
            const int64_t l1 = M1.lev[jj] + 1;
            const int64_t ysz = 2 * (int64_t)M0.lev[jj - 1] * l1 + ADJ_SLACK;
            const int64_t zsz = 4 * (int64_t)M0.lev[jj] * l1;
            bneed = std::max(bneed, std::max(prevZ + ysz, zsz + ysz));
            bneed = std::max(bneed, zsz + ADJ_SLACK * l1);
            prevZ = zsz;
        }
    }
    if (!stencils_inside(g, b, bp.k0, bp.jhi))
        return fail(h, PC_ERR_UNSUPPORTED, "internal: stencil of band %d outside its transform range", b);
    need = round_up(need, (int64_t)(16 / es));
    bneed = (bneed < 0) ? need : round_up(bneed, (int64_t)(16 / es));
    const int lft = (g.d == 2) ? lf_template(g.Lf) : g.Lf;
    int filt = 2 * lft + ((bp.k0 > 0) ? wav_len(bp.k0, g.Lf) : 0);
    filt = (int)round_up(filt, (int64_t)(16 / es));
    int rpc = std::max(1, 256 / gt);
    auto smem_of = [&](int rpcv, int64_t ar) {
        return (size_t)filt * es + round_up((int64_t)rpcv * META_INTS * 4, 16) + (size_t)rpcv * ar * es;
    };
    const int64_t amax = std::max(need, bneed);
    while (rpc > 1 && smem_of(rpc, amax) > 110 * 1024) rpc /= 2;
    if (smem_of(rpc, amax) > 227 * 1024)
        return fail(h, PC_ERR_UNSUPPORTED, "band %d needs %zu bytes of shared memory per row", b, smem_of(rpc, amax));
    bp.cfg.b = b;
    bp.cfg.row0 = 0;
    bp.cfg.rows = bp.rows;
    bp.cfg.gt = gt;
    bp.cfg.rpc = rpc;
    bp.cfg.batch = batch;
    bp.cfg.arena = (int)need;
    bp.cfg.filt = filt;
    bp.smem = smem_of(rpc, need);
    bp.cfg_b = bp.cfg;
    bp.cfg_b.arena = (int)bneed;
    bp.smem_b = smem_of(rpc, bneed);
    *out = bp;
    return PC_OK;
}

pc_status plan_bands(pc_op* h)
{
    Geo g = geo_of(&h->desc);
    h->plan.clear();
    for (int b = 0; b < g.nb; ++b) {
        BandPlan bp;
        pc_status st = plan_band(h, g, b, 0, &bp);
        if (st != PC_OK) return st;
        h->plan.push_back(bp);
    }
    return PC_OK;
}

template <typename T>
OpDev<T> make_opdev(pc_op* h)
{
    OpDev<T> o{};
    const pc_desc& D = h->desc;
    o.d = D.dim;
    o.n = D.n;
    o.L = D.levels;
    o.Lf = h->Lf;
    o.r = D.radius;
    o.m = D.m;
    o.gap = D.gap;
    o.order = D.order;
    o.nb = h->nb;
    o.N = h->N;
    o.u = (const T*)h->u_d;
    o.v = (const T*)h->v_d;
    o.taps = (const T*)h->tapsT_d;
    o.wav = (const T*)h->wavT_d;
    for (int i = 0; i < MAXL + 2; ++i) o.wofs[i] = h->wofs[i];
    o.F = (const T*)h->F_d;
    for (int b = 0; b < h->nb; ++b) o.Foff[b] = h->fd.band[b].Foff;
    o.row_ptr = h->row_ptr_d;
    o.theta = (T*)h->theta_d;
    o.theta16 = h->theta16_d;
    o.masks = h->masks_d;
    o.mwords = h->mwords;
    o.ts0 = h->ts0;
    o.ts1 = h->ts1;
    o.tpa0 = h->tpa0;
    o.tpa1 = h->tpa1;
    o.err = h->err_d;
    o.wl = h->wl_d;
    o.sf = (h->desc.dim == 2) ? (T*)h->S_d : nullptr;
    for (int b = 0; b < h->nb; ++b) o.Soff[b] = h->bd.band[b].Soff;
    o.wl_slots = h->wl_slots;
    return o;
}

template <typename T, int DIM>
pc_status set_smem_attr()
{
    static bool done = false;
    if (!done) {
        if ((DIM == 1 &&
             cudaFuncSetAttribute(k_assemble1d<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024) !=
                 cudaSuccess) ||
            cudaFuncSetAttribute(k_backward<T, DIM>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024) !=
                cudaSuccess)
            return PC_ERR_CUDA;
        done = true;
    }
    return PC_OK;
}

template <typename T, int LF>
pc_status launch_asm2d_lf(pc_op* h, const OpDev<T>& od, const BandPlan& bp, int ctas, int threads, cudaStream_t st)
{
    static bool attr = false;
    if (!attr) {
        if (cudaFuncSetAttribute(k_assemble2d<T, LF>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024) !=
            cudaSuccess)
            return fail(h, PC_ERR_CUDA, "cudaFuncSetAttribute failed");
        attr = true;
    }
    k_assemble2d<T, LF><<<ctas, threads, bp.smem, st>>>(od, bp.cfg);
    return PC_OK;
}

template <typename T>
pc_status launch_asm2d(pc_op* h, const OpDev<T>& od, const BandPlan& bp, int ctas, int threads, cudaStream_t st)
{
    switch (lf_template(h->Lf)) {
        case 2: return launch_asm2d_lf<T, 2>(h, od, bp, ctas, threads, st);
        case 4: return launch_asm2d_lf<T, 4>(h, od, bp, ctas, threads, st);
        case 8: return launch_asm2d_lf<T, 8>(h, od, bp, ctas, threads, st);
        default: return launch_asm2d_lf<T, 20>(h, od, bp, ctas, threads, st);
    }
}

template <typename T>
pc_status prepare_t(pc_op* h, cudaStream_t st)
{
    const pc_desc& D = h->desc;
    // taps in T and the FP64 cascade of the base wavelets
    k_taps<T><<<1, 64, 0, st>>>(h->taps64_d, h->Lf, (T*)h->tapsT_d);
    k_base_wavelets<<<1, 256, 0, st>>>(h->taps64_d, h->Lf, D.levels, h->wav64_d);
    k_cast<T><<<std::max(1, std::min(1024, (h->wav_total + 255) / 256)), 256, 0, st>>>(h->wav64_d, (T*)h->wavT_d,
                                                                                      h->wav_total);
    // filtered base wavelets
    {
        int maxU = 0, maxR = 0;
        const int K0 = (D.dim == 2) ? h->K : 1;
        for (int b = 0; b < h->nb; ++b) {
            maxU = std::max(maxU, K0 * h->fd.band[b].U1);
            maxR = std::max(maxR, h->fd.band[b].R0 * h->fd.band[b].R1);
        }
        // each block stages its gathered inputs (pass 1: the kernel stencil and the band's 1-D
        // factor; pass 2: the factor) in shared memory when they fit 48 KB, else reads them from
        // global memory
        const int lenmax = wav_len(D.levels, h->Lf);
        const int Ku = (D.dim == 2) ? h->K * h->K : h->K;
        const size_t sm1 = sizeof(T) * (size_t)(Ku + lenmax), sm2 = sizeof(T) * (size_t)lenmax;
        const int st1 = sm1 <= 48 * 1024, st2 = sm2 <= 48 * 1024;
        dim3 g1((maxU + 127) / 128, h->nb * D.m), g2((maxR + 127) / 128, h->nb * D.m);
        k_filtered_pass1<T><<<g1, 128, st1 ? sm1 : 0, st>>>(h->fd, (const T*)h->u_d, (const T*)h->wavT_d,
                                                           (T*)h->G_d, st1);
        k_filtered_pass2<T><<<g2, 128, st2 ? sm2 : 0, st>>>(h->fd, (const T*)h->wavT_d, (const T*)h->G_d,
                                                           (T*)h->F_d, st2);
    }
    // window tile masks
    k_tile_masks<T><<<h->tpa0 * h->tpa1, 256, 0, st>>>((const T*)h->v_d, D.dim, D.n, D.m, h->ts0, h->ts1, h->tpa1,
                                                       h->mwords, h->masks_d);
    count_launch(6);
    PC_CUDA(h, cudaGetLastError());
    return PC_OK;
}

// Stage 1 of every 2-D row (k_s_tiles) into the s scratch, before the row kernels.
template <typename T>
pc_status s_rows_t(pc_op* h, const OpDev<T>& od, cudaStream_t st, const OpDev<T>* od_dev = nullptr)
{
    if (h->desc.dim != 2 || !h->S_d) return PC_OK;
    if (!od_dev) {
        PC_CUDA(h, cudaMemcpyAsync(h->od_d, &od, sizeof(od), cudaMemcpyHostToDevice, st));
        od_dev = (const OpDev<T>*)h->od_d;
    }
    // tiles of 8 consecutive rows along axis 1 (fewer in bands narrower than that)
    STiles tl{};
    tl.T = 8;
    int tiles = 0;
    for (int b = 0; b < h->nb; ++b) {
        const Band B = band_info(2, h->desc.n, h->desc.levels, b);
        tl.tile_off[b] = tiles;
        tiles += B.nj * ((B.nj + tl.T - 1) / tl.T);
    }
    tl.tile_off[h->nb] = tiles;
    k_s_tiles<T><<<tiles, 256, 0, st>>>(od_dev, tl);
    count_launch();
    PC_CUDA(h, cudaGetLastError());
    return PC_OK;
}

template <typename T>
pc_status assemble_t(pc_op* h, cudaStream_t st, int stage_mask)
{
    const pc_desc& D = h->desc;
    if (stage_mask & 1) {
        pc_status ps = prepare_t<T>(h, st);
        if (ps != PC_OK) return ps;
        h->prepared = true;
    }
    if (!(stage_mask & 2)) return PC_OK;
    if (!h->prepared) return fail(h, PC_ERR_INVALID_ARG, "assembly stage 1 before stage 0");
    if constexpr (std::is_same<T, float>::value) {
        if (h->q_items_d && h->q_smem <= 110 * 1024) {
            // one persistent launch over all row bands, longest work items first
            const OpDev<float> od = make_opdev<float>(h);
            PC_CUDA(h, cudaMemcpyAsync(h->q_op_d, &od, sizeof(od), cudaMemcpyHostToDevice, st));
            pc_status sp = s_rows_t<float>(h, od, st, h->q_op_d);
            if (sp != PC_OK) return sp;
            PC_CUDA(h, cudaMemsetAsync(h->q_counter_d, 0, sizeof(int), st));
            queue_kernel(h->q_kind)<<<h->q_grid, 256, h->q_smem, st>>>(h->q_op_d, h->q_items_d, h->q_nitems,
                                                                       h->q_counter_d);
            count_launch();
            PC_CUDA(h, cudaGetLastError());
            h->assembled = true;
            h->theta_gen++;
            return PC_OK;
        }
    }
    // one launch per row band
    OpDev<T> od = make_opdev<T>(h);
    {
        pc_status sp = s_rows_t<T>(h, od, st);
        if (sp != PC_OK) return sp;
    }
    for (const BandPlan& bp : h->plan) {
        const int ctas = (bp.rows + bp.cfg.rpc - 1) / bp.cfg.rpc;
        const int threads = bp.cfg.gt * bp.cfg.rpc;
        if (D.dim == 1) {
            if (set_smem_attr<T, 1>() != PC_OK) return fail(h, PC_ERR_CUDA, "cudaFuncSetAttribute failed");
            k_assemble1d<T><<<ctas, threads, bp.smem, st>>>(od, bp.cfg);
        } else {
            pc_status ls = launch_asm2d<T>(h, od, bp, ctas, threads, st);
            if (ls != PC_OK) return ls;
        }
        count_launch();
    }
    PC_CUDA(h, cudaGetLastError());
    h->assembled = true;
    h->theta_gen++;
    return PC_OK;
}

template <typename TA>
OpDev<TA> apply_od(const pc_op* h)
{
    OpDev<TA> od{};
    const pc_desc& D = h->desc;
    od.d = D.dim;
    od.n = D.n;
    od.L = D.levels;
    od.Lf = h->Lf;
    od.r = D.radius;
    od.gap = D.gap;
    od.nb = h->nb;
    od.N = h->N;
    od.row_ptr = h->row_ptr_d;
    return od;
}

template <typename T>
pc_status dev_alloc(pc_op* h, T** p, size_t bytes);

// Column-block descriptors (built once per handle; they depend on the pattern only).
template <typename TA>
pc_status ensure_block_desc(pc_op* h, cudaStream_t st)
{
    if (h->bdesc_d) return PC_OK;
    const pc_desc& D = h->desc;
    int kmax = 1;
    for (int b = 0; b < h->nb; ++b) {
        int k = 0;
        for (int b2 = 0; b2 < h->nb; ++b2) k += block_kept(D.dim, D.n, D.levels, D.gap, b, b2) ? 1 : 0;
        kmax = std::max(kmax, k);
    }
    pc_status e = dev_alloc(h, &h->bdesc_d, sizeof(unsigned long long) * (size_t)h->N * kmax);
    if (e != PC_OK) return e;
    if ((e = dev_alloc(h, &h->boff_d, sizeof(unsigned) * (size_t)h->N * kmax)) != PC_OK) return e;
    h->bdesc_stride = kmax;
    OpDev<TA> od = apply_od<TA>(h);
    od.nb = h->nb;
    k_block_desc<TA><<<(int)((h->N + 255) / 256), 256, 0, st>>>(od, h->bdesc_d, h->boff_d, kmax);
    count_launch();
    PC_CUDA(h, cudaGetLastError());
    return PC_OK;
}

// Transposed copy of the stored values for the current assembly (built on first use after
// each assembly; descriptors must exist).
template <typename T>
pc_status ensure_thetaT(pc_op* h, cudaStream_t st)
{
    if (h->thetaT_d && h->thetaT_gen == h->theta_gen) return PC_OK;
    if (!h->thetaT_d) {
        T* p = nullptr;
        pc_status e = dev_alloc(h, &p, sizeof(T) * (size_t)h->nnz);
        if (e != PC_OK) return e;
        h->thetaT_d = p;
    }
    OpDev<T> od = apply_od<T>(h);
    od.nb = h->bdesc_stride;
    od.err = h->err_d;
    k_transpose_theta<T><<<(int)((h->N * 32 + 255) / 256), 256, 0, st>>>(od, h->bdesc_d, h->boff_d, h->nb,
                                                                         (const T*)h->theta_d, (T*)h->thetaT_d);
    count_launch();
    PC_CUDA(h, cudaGetLastError());
    h->thetaT_gen = h->theta_gen;
    return PC_OK;
}

// One column: y = Theta x - sub (adjoint = false; sub may be null) or y = Theta^T x
// (adjoint = true).
// With use_T (values of the handle's own type only) a product that would scatter over the
// stored rows gathers over the rows of the transposed copy instead: no atomics, and the same
// cost as the stored direction.
template <typename TV, typename TA, bool SQ>
pc_status apply1_t(pc_op* h, const TV* vals, const TA* x, TA* y, const TA* sub, bool adjoint, cudaStream_t st,
                   bool use_T = false)
{
    pc_status e = ensure_block_desc<TA>(h, st);
    if (e != PC_OK) return e;
    OpDev<TA> od = apply_od<TA>(h);
    od.nb = h->bdesc_stride;
    bool transpose = (h->desc.order == PC_ORDER_CONV_THEN_MULT) != adjoint;
    if constexpr (std::is_same<TV, TA>::value) {
        if (transpose && use_T) {
            if ((e = ensure_thetaT<TA>(h, st)) != PC_OK) return e;
            vals = (const TV*)h->thetaT_d;
            transpose = false;
        }
    }
    if (transpose) {
        if (sub) return fail(h, PC_ERR_INVALID_ARG, "internal: subtraction on a scattered product");
        k_zero_rows<TA><<<(int)((h->N + 255) / 256), 256, 0, st>>>(y, h->N, 1, 0, 1);
        k_apply1<TV, TA, SQ, 1, 32><<<(int)((h->N * 32 + 255) / 256), 256, 0, st>>>(od, h->bdesc_d, vals, x, y,
                                                                                   nullptr);
        count_launch(2);
    } else {
        // the fewest lanes per row that still give three quarters of a wave of warps (64 per SM)
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int64_t want = (int64_t)std::max(sms, 1) * 64 * 32 * 3 / 4;
        if (h->N * 8 >= want)
            k_apply1<TV, TA, SQ, 0, 8><<<(int)((h->N * 8 + 255) / 256), 256, 0, st>>>(od, h->bdesc_d, vals, x, y, sub);
        else if (h->N * 16 >= want)
            k_apply1<TV, TA, SQ, 0, 16><<<(int)((h->N * 16 + 255) / 256), 256, 0, st>>>(od, h->bdesc_d, vals, x, y,
                                                                                        sub);
        else
            k_apply1<TV, TA, SQ, 0, 32><<<(int)((h->N * 32 + 255) / 256), 256, 0, st>>>(od, h->bdesc_d, vals, x, y,
                                                                                        sub);
        count_launch();
    }
    PC_CUDA(h, cudaGetLastError());
    return PC_OK;
}

// y = Theta x (adjoint = false) or y = Theta^T x; SQ squares the stored values first.
template <typename TV, typename TA, bool SQ = false>
pc_status apply_t(pc_op* h, const TV* vals, const TA* x, TA* y, int nrhs, int ldx, int ldy, cudaStream_t st,
                  bool adjoint = false)
{
    OpDev<TA> od{};
    const pc_desc& D = h->desc;
    od.d = D.dim;
    od.n = D.n;
    od.L = D.levels;
    od.Lf = h->Lf;
    od.r = D.radius;
    od.gap = D.gap;
    od.nb = h->nb;
    od.N = h->N;
    od.row_ptr = h->row_ptr_d;
    const int transpose = (D.order == PC_ORDER_CONV_THEN_MULT) != adjoint;
    const int64_t warps = h->N;
    const int blocks = (int)((warps * 32 + 255) / 256);
    // tensor-core path: BF16 values, paper order, groups of 16 right-hand sides
    if constexpr (std::is_same<TV, __nv_bfloat16>::value && std::is_same<TA, float>::value) {
        if (!SQ && !transpose && nrhs >= 16 && h->xsplit_d) {
            TcApply tp{};
            tp.d = D.dim;
            tp.n = D.n;
            tp.L = D.levels;
            tp.Lf = h->Lf;
            tp.r = D.radius;
            tp.gap = D.gap;
            tp.nb = h->nb;
            tp.N = h->N;
            tp.row_ptr = h->row_ptr_d;
            int tiles = 0;
            for (int b = 0; b < h->nb; ++b) {
                tp.tile_off[b] = tiles;
                const Band B = band_info(D.dim, D.n, D.levels, b);
                tiles += ((D.dim == 2) ? B.nj : 1) * ((B.nj + 15) / 16);
            }
            tp.tile_off[h->nb] = tiles;
            int c = 0;
            for (; nrhs - c >= 16; c += 16) {
                k_split_x<<<(int)((h->N * 16 + 255) / 256), 256, 0, st>>>(x, ldx, c, h->N, h->xsplit_d);
                k_apply_tc<<<tiles, 128, 0, st>>>(tp, vals, h->xsplit_d, y, ldy, c);
                count_launch(2);
            }
            PC_CUDA(h, cudaGetLastError());
            if (c == nrhs) return PC_OK;
            x += c;
            y += c;
            nrhs -= c;
        }
    }
    // vectorised path: paper order, FP32 accumulation, 16-byte aligned x/y with ldx, ldy % 4 == 0;
    // right-hand sides in groups of 16, 8 or 4, a remainder below 4 by the scalar kernel
    if constexpr (std::is_same<TA, float>::value) {
        const bool vec = !SQ && !transpose && ((uintptr_t)x % 16 == 0) && ((uintptr_t)y % 16 == 0) && ldx % 4 == 0 &&
                         ldy % 4 == 0;
        if (vec) {
            int c = 0;
            while (nrhs - c >= 4) {
                const int rem = nrhs - c;
                if (rem >= 16) {
                    k_apply_vec<TV, 16><<<blocks, 256, 0, st>>>(od, vals, x, ldx, y, ldy, c);
                    c += 16;
                } else if (rem >= 8) {
                    k_apply_vec<TV, 8><<<blocks, 256, 0, st>>>(od, vals, x, ldx, y, ldy, c);
                    c += 8;
                } else {
                    k_apply_vec<TV, 4><<<blocks, 256, 0, st>>>(od, vals, x, ldx, y, ldy, c);
                    c += 4;
                }
                count_launch();
            }
            PC_CUDA(h, cudaGetLastError());
            if (c == nrhs) return PC_OK;
            x += c;
            y += c;
            nrhs -= c;
        }
    }
    if (nrhs == 1 && ldx == 1 && ldy == 1) return apply1_t<TV, TA, SQ>(h, vals, x, y, nullptr, adjoint, st);
    for (int c0 = 0; c0 < nrhs; c0 += 16) {
        const int nr = std::min(16, nrhs - c0);
        if (transpose) {
            k_zero_rows<TA><<<(int)((h->N * nr + 255) / 256), 256, 0, st>>>(y, h->N, ldy, c0, nr);
            count_launch();
        }
        count_launch();
        if (nr == 1)
            k_apply<TV, TA, 1, SQ><<<blocks, 256, 0, st>>>(od, vals, x, ldx, y, ldy, c0, nr, transpose);
        else if (nr <= 4)
            k_apply<TV, TA, 4, SQ><<<blocks, 256, 0, st>>>(od, vals, x, ldx, y, ldy, c0, nr, transpose);
        else
            k_apply<TV, TA, 16, SQ><<<blocks, 256, 0, st>>>(od, vals, x, ldx, y, ldy, c0, nr, transpose);
    }
    PC_CUDA(h, cudaGetLastError());
    return PC_OK;
}

template <typename T>
pc_status dev_alloc(pc_op* h, T** p, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc((void**)p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        return fail(h, PC_ERR_OOM, "cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
    }
    h->dev_bytes += (int64_t)bytes;
    return PC_OK;
}

// Backward kernels with caller-chosen scratch: dF (Ftotal elements, zeroed here) and dG
// (Gtotal elements, fully overwritten).
template <typename T, int LF>
pc_status launch_bwd2d_lf(pc_op* h, const OpDev<T>& od, const BandPlan& bp, int ctas, int threads, const T* G, T* S,
                          int64_t Sband, unsigned long long* amask, cudaStream_t st)
{
    static bool attr = false;
    if (!attr) {
        if (cudaFuncSetAttribute(k_backward2d<T, LF>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024) !=
            cudaSuccess)
            return fail(h, PC_ERR_CUDA, "cudaFuncSetAttribute failed");
        attr = true;
    }
    k_backward2d<T, LF><<<ctas, threads, bp.smem_b, st>>>(od, bp.cfg_b, G, S, Sband, amask);
    return PC_OK;
}

template <typename T>
pc_status launch_bwd2d(pc_op* h, const OpDev<T>& od, const BandPlan& bp, int ctas, int threads, const T* G, T* S,
                       int64_t Sband, unsigned long long* amask, cudaStream_t st)
{
    switch (lf_template(h->Lf)) {
        case 2: return launch_bwd2d_lf<T, 2>(h, od, bp, ctas, threads, G, S, Sband, amask, st);
        case 4: return launch_bwd2d_lf<T, 4>(h, od, bp, ctas, threads, G, S, Sband, amask, st);
        case 8: return launch_bwd2d_lf<T, 8>(h, od, bp, ctas, threads, G, S, Sband, amask, st);
        default: return launch_bwd2d_lf<T, 20>(h, od, bp, ctas, threads, G, S, Sband, amask, st);
    }
}

// Backward kernels with caller-chosen scratch: dF (Ftotal elements, zeroed here), dG (Gtotal
// elements, fully overwritten) and, for 2-D operators, optionally S (Stotal elements, fully
// overwritten).  With S: the three-phase path (dL/ds per row to S, then dv by a per-pixel
// gather and dF by per-band reductions).  Without S: dv and dF by atomics from the rows.
template <typename T>
pc_status backward_core(pc_op* h, const T* G, T* du, T* dv, T* dF, T* dG, cudaStream_t st, T* S = nullptr,
                        unsigned long long* amask = nullptr)
{
    const pc_desc& D = h->desc;
    pc_status ps = prepare_t<T>(h, st);  // filtered wavelets recomputed from the current u
    if (ps != PC_OK) return ps;
    PC_CUDA(h, cudaMemsetAsync(dF, 0, h->esz * h->Ftotal, st));
    OpDev<T> od = make_opdev<T>(h);
    if (D.dim == 2 && S) {
        // phase 3 sums over the window lists when they exist: no active-term masks needed then
        const bool dF_wl = h->wl_d && (size_t)D.m * 128 * h->esz <= 48 * 1024;
        if (dF_wl) amask = nullptr;
        bool queued = false;
        if constexpr (std::is_same<T, float>::value) {
            if (h->q_items_b_d && h->q_smem_b <= 110 * 1024) {
                // phase 1 through the operator's work queue: one launch over all row bands
                const BwdQueueKernel kq = bwd_queue_kernel(h->q_kind);
                PC_CUDA(h, cudaFuncSetAttribute(kq, cudaFuncAttributeMaxDynamicSharedMemorySize, 110 * 1024));
                const OpDev<float> odq = make_opdev<float>(h);
                PC_CUDA(h, cudaMemcpyAsync(h->q_op_d, &odq, sizeof(odq), cudaMemcpyHostToDevice, st));
                PC_CUDA(h, cudaMemsetAsync(h->q_counter_d, 0, sizeof(int), st));
                BwdQueue bq{};
                bq.G = G;
                bq.S = S;
                bq.amask = amask;
                for (int b = 0; b < h->nb; ++b) bq.Soff[b] = h->bd.band[b].Soff;
                kq<<<persistent_grid(kq, h->q_smem_b), 256, h->q_smem_b, st>>>(h->q_op_d, h->q_items_b_d,
                                                                               h->q_nitems, h->q_counter_d, bq);
                count_launch();
                queued = true;
            }
        }
        if (!queued)
            for (const BandPlan& bp : h->plan) {
                const int ctas = (bp.rows + bp.cfg.rpc - 1) / bp.cfg.rpc;
                const int threads = bp.cfg.gt * bp.cfg.rpc;
                pc_status ls = launch_bwd2d<T>(h, od, bp, ctas, threads, G, S, h->bd.band[bp.b].Soff, amask, st);
                if (ls != PC_OK) return ls;
                count_launch();
            }
        constexpr int KC = 8;
        if constexpr (std::is_same<T, float>::value) {
            // term-contiguous copy of F (in the tail of the dL/dG scratch), then float4 gathers
            float* FT = (float*)h->dG_d + (h->Gtotal + 3) / 4 * 4;  // 16-byte aligned
            int maxRR = 0;
            for (int b = 0; b < h->nb; ++b) maxRR = std::max(maxRR, h->bd.band[b].R0 * h->bd.band[b].R1);
            k_transpose_F<<<dim3((maxRR + 255) / 256, h->nb), 256, 0, st>>>(h->bd, (const float*)h->F_d, FT);
            // 32 x 8 pixel tiles (16 x 16 below 32 pixels a side); 16 terms per thread when that
            // still gives >= 2048 blocks (each dL/ds value is loaded once per group of terms), else 8
            const int tiles32 = ((D.n + 31) / 32) * ((D.n + 7) / 8), zc4 = (D.m + 15) / 16, zc2 = (D.m + 7) / 8;
            if (D.n >= 32 && D.m > 8 && tiles32 * zc4 >= 2048)
                k_bwd_dv4<4, 32><<<dim3((D.n + 31) / 32 * zc4, (D.n + 7) / 8, 1), dim3(32, 8), 0, st>>>(h->bd, FT, S, dv);
            else if (D.n >= 32)
                k_bwd_dv4<2, 32><<<dim3((D.n + 31) / 32 * zc2, (D.n + 7) / 8, 1), dim3(32, 8), 0, st>>>(h->bd, FT, S, dv);
            else
                k_bwd_dv4<2, 16><<<dim3((D.n + 15) / 16 * zc2, (D.n + 15) / 16, 1), dim3(16, 16), 0, st>>>(h->bd, FT, S,
                                                                                                      dv);
            count_launch(2);
        } else {
            k_bwd_dv<T, KC><<<dim3((D.n + 15) / 16, (D.n + 15) / 16, (D.m + KC - 1) / KC), dim3(16, 16), 0, st>>>(
                h->bd, (const T*)h->F_d, S, dv);
            count_launch();
        }
        {
            // one launch over all bands: blocks (band, 128 region positions, a chunk of rows); larger
            // operators take longer chunks (fewer blocks and fewer atomic adds per dL/dF entry)
            const int chunk = h->N >= ((int64_t)1 << 20) ? 128 : h->N >= ((int64_t)1 << 16) ? 64 : 32;
            int offs[MAXB + 1];
            int tot = 0;
            for (int b = 0; b < h->nb; ++b) {
                const BwdBand& B = h->bd.band[b];
                offs[b] = tot;
                tot += ((B.R0 * B.R1 + 127) / 128) * ((B.nj * B.nj + chunk - 1) / chunk);
            }
            offs[h->nb] = tot;
            PC_CUDA(h, cudaMemcpyAsync(h->dfoff_d, offs, sizeof(int) * (h->nb + 1), cudaMemcpyHostToDevice, st));
            const size_t acc_bytes = (size_t)D.m * 128 * h->esz;
            if (dF_wl)
                k_bwd_dF_wl<T><<<tot, 128, acc_bytes, st>>>(h->bd, (const WSlot<T>*)h->wl_d, h->wl_slots, S, dF,
                                                           h->dfoff_d, chunk);
            else
                k_bwd_dF<T, 16><<<dim3(tot, 1, (D.m + 15) / 16), 128, 0, st>>>(h->bd, (const T*)h->v_d, S, amask,
                                                                              h->mwords, dF, h->dfoff_d, chunk);
            count_launch();
        }
    } else {
        PC_CUDA(h, cudaMemsetAsync(dv, 0, h->esz * D.m * h->N, st));
        for (const BandPlan& bp : h->plan) {
            const int ctas = (bp.rows + bp.cfg.rpc - 1) / bp.cfg.rpc;
            const int threads = bp.cfg.gt * bp.cfg.rpc;
            if (D.dim == 1) {
                if (set_smem_attr<T, 1>() != PC_OK) return fail(h, PC_ERR_CUDA, "cudaFuncSetAttribute failed");
                k_backward<T, 1><<<ctas, threads, bp.smem_b, st>>>(od, bp.cfg_b, G, dv, dF);
            } else {
                if (set_smem_attr<T, 2>() != PC_OK) return fail(h, PC_ERR_CUDA, "cudaFuncSetAttribute failed");
                k_backward<T, 2><<<ctas, threads, bp.smem_b, st>>>(od, bp.cfg_b, G, dv, dF);
            }
            count_launch();
        }
    }
    int maxU = 0;
    const int K0 = (D.dim == 2) ? h->K : 1;
    for (int b = 0; b < h->nb; ++b) maxU = std::max(maxU, K0 * h->fd.band[b].U1);
    k_dfilt_pass2<T><<<dim3((maxU + 127) / 128, h->nb * D.m), 128, 0, st>>>(h->fd, (const T*)h->wavT_d, dF, dG);
    k_dfilt_pass1<T><<<(D.m * h->Ku + 127) / 128, 128, 0, st>>>(h->fd, (const T*)h->wavT_d, dG, du);
    count_launch(2);
    PC_CUDA(h, cudaGetLastError());
    return PC_OK;
}

// pc_backward: scratch owned by the handle, allocated on first use.
template <typename T>
pc_status backward_t(pc_op* h, const T* G, T* du, T* dv, cudaStream_t st)
{
    if (!h->dF_d) {
        pc_status a;
        if ((a = dev_alloc(h, &h->dF_d, h->esz * h->Ftotal)) != PC_OK) return a;
        if ((a = dev_alloc(h, &h->dG_d, h->esz * ((h->Gtotal + 3) / 4 * 4 + h->FTtotal))) != PC_OK) return a;
        if (h->desc.dim == 2 && !h->S_d && (a = dev_alloc(h, &h->S_d, h->esz * h->Stotal)) != PC_OK) return a;
        if (h->desc.dim == 2 &&
            (a = dev_alloc(h, &h->amask_d, sizeof(unsigned long long) * h->N * h->mwords)) != PC_OK)
            return a;
        if (h->desc.dim == 2 && (a = dev_alloc(h, &h->dfoff_d, sizeof(int) * (MAXB + 1))) != PC_OK) return a;
    }
    return backward_core<T>(h, G, du, dv, (T*)h->dF_d, (T*)h->dG_d, st, (T*)h->S_d, h->amask_d);
}

// Scratch of pc_backward_noalloc: one static device array per GPU that loads the library.
// Host code must not use the symbol as an address: its device address comes from
// cudaGetSymbolAddress, looked up once per device (with that device current) and cached.
static __device__ __align__(256) unsigned char g_noalloc_scratch[PC_NOALLOC_SCRATCH_BYTES];
constexpr int kMaxDevices = 256;
std::mutex g_noalloc_mu;
void* g_noalloc_addr[kMaxDevices] = {};

pc_status noalloc_scratch(pc_op* h, void** out)
{
    int dev = -1;
    PC_CUDA(h, cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(h, PC_ERR_UNSUPPORTED, "device index %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return fail(h, PC_ERR_CUDA, "cudaGetSymbolAddress of the static scratch failed on device %d: %s", dev,
                        cudaGetErrorString(e));
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return PC_OK;
}

template <typename T>
pc_status backward_noalloc_t(pc_op* h, const T* G, T* du, T* dv, cudaStream_t st)
{
    const size_t fbytes = h->esz * (size_t)h->Ftotal;
    const size_t goff = (fbytes + 255) / 256 * 256;
    const size_t need = goff + h->esz * (size_t)h->Gtotal;
    if (need > (size_t)PC_NOALLOC_SCRATCH_BYTES)
        return fail(h, PC_ERR_UNSUPPORTED,
                    "pc_backward_noalloc: this operator needs %zu bytes of scratch, the static array holds %u",
                    need, (unsigned)PC_NOALLOC_SCRATCH_BYTES);
    void* base = nullptr;
    pc_status st0 = noalloc_scratch(h, &base);
    if (st0 != PC_OK) return st0;
    T* dF = (T*)base;                             // zeroed by backward_core
    T* dG = (T*)((unsigned char*)base + goff);    // fully overwritten
    return backward_core<T>(h, G, du, dv, dF, dG, st);
}

// Window lists (rebuilt whenever the windows change): count the most nonzero windows at a
// pixel (synchronous read of one int), grow the list if needed, fill it.
template <typename T>
pc_status build_window_list_t(pc_op* h, cudaStream_t st)
{
    const pc_desc& D = h->desc;
    if (!h->cnt_d) {
        pc_status a = dev_alloc(h, &h->cnt_d, sizeof(int));
        if (a != PC_OK) return a;
    }
    const int blocks = (int)((h->N + 255) / 256);
    PC_CUDA(h, cudaMemsetAsync(h->cnt_d, 0, sizeof(int), st));
    k_window_count<T><<<blocks, 256, 0, st>>>((const T*)h->v_d, D.m, h->N, h->cnt_d);
    count_launch();
    int slots = 0;
    PC_CUDA(h, cudaMemcpyAsync(&slots, h->cnt_d, sizeof(int), cudaMemcpyDeviceToHost, st));
    PC_CUDA(h, cudaStreamSynchronize(st));
    slots = std::max(slots, 1);
    if (slots > h->wl_slots || !h->wl_d) {
        if (h->wl_d) {
            cudaDeviceSynchronize();  // a batch on another stream may still read the old list
            cudaFree(h->wl_d);
            h->dev_bytes -= (int64_t)sizeof(WSlot<T>) * h->wl_slots * h->N;
            h->wl_d = nullptr;
        }
        pc_status a = dev_alloc(h, &h->wl_d, sizeof(WSlot<T>) * (size_t)slots * h->N);
        if (a != PC_OK) return a;
    }
    h->wl_slots = slots;
    k_window_list<T><<<blocks, 256, 0, st>>>((const T*)h->v_d, D.m, h->N, slots, (WSlot<T>*)h->wl_d);
    count_launch();
    PC_CUDA(h, cudaGetLastError());
    return PC_OK;
}

pc_status build_window_list(pc_op* h, cudaStream_t st)
{
    if (h->desc.dim != 2) return PC_OK;  // the 1-D rows sum over the active terms of their region
    return h->desc.precision == PC_FP64 ? build_window_list_t<double>(h, st) : build_window_list_t<float>(h, st);
}

void free_all(pc_op* h)
{
    void* ptrs[] = {h->u_d,  h->v_d,        h->taps64_d,  h->wav64_d,  h->tapsT_d, h->wavT_d, h->F_d,
                    h->G_d,  h->dF_d, h->dG_d, h->S_d, h->amask_d, h->wl_d, h->cnt_d, h->dfoff_d, h->q_items_d, h->q_items_b_d, h->q_op_d, h->q_counter_d, h->row_ptr_d,  h->theta_d,   h->theta16_d, h->xsplit_d, h->od_d, h->masks_d, h->err_d, h->fista_d, h->bdesc_d, h->boff_d, h->thetaT_d};
    for (void* p : ptrs)
        if (p) cudaFree(p);
}

// Work items of one operator: every row band split into runs of rows of similar cost
// (region arena + stored entries per row), with the band's plan.
struct ItemCand {
    double cost;
    BatchItem it;
};

void make_items(pc_op* h, int op_index, std::vector<ItemCand>* out, size_t* smem, bool adjoint = false)
{
    for (const BandPlan& bp : h->plan) {
        const Band B = band_info(h->desc.dim, h->desc.n, h->desc.levels, bp.b);
        const double entries = (double)(h->row_ptr_h[B.off + bp.rows] - h->row_ptr_h[B.off]) / bp.rows;
        const double row_cost = (double)bp.cfg.arena + entries;
        int per = (int)std::max(1.0, std::floor(60000.0 / row_cost));
        per = std::max(bp.cfg.rpc, (per / bp.cfg.rpc) * bp.cfg.rpc);
        for (int r0 = 0; r0 < bp.rows; r0 += per) {
            ItemCand c;
            c.it.op = op_index;
            c.it.dim = h->desc.dim;
            c.it.lft = (h->desc.dim == 2) ? lf_template(h->Lf) : h->Lf;
            c.it.pad = 0;
            c.it.cfg = adjoint ? bp.cfg_b : bp.cfg;
            c.it.cfg.row0 = r0;
            c.it.cfg.rows = std::min(per, bp.rows - r0);
            c.cost = row_cost * c.it.cfg.rows;
            out->push_back(c);
            *smem = std::max(*smem, adjoint ? bp.smem_b : bp.smem);
        }
    }
}

// (Re)builds the single-operator queue from the current plan.
pc_status build_queue(pc_op* h)
{
    if (h->desc.precision != PC_FP32) return PC_OK;
    pc_status a;
    for (int adj = 0; adj < 2; ++adj) {
        // forward and adjoint items in the same order (sorted by the forward cost)
        std::vector<ItemCand> cands;
        size_t smem = 0;
        make_items(h, 0, &cands, &smem, adj == 1);
        std::stable_sort(cands.begin(), cands.end(),
                         [](const ItemCand& x, const ItemCand& y) { return x.cost > y.cost; });
        std::vector<BatchItem> items;
        for (const ItemCand& c : cands) items.push_back(c.it);
        if (items.empty()) return PC_OK;
        BatchItem*& dst = adj ? h->q_items_b_d : h->q_items_d;
        if (dst) {
            cudaFree(dst);
            dst = nullptr;
        }
        if ((a = dev_alloc(h, &dst, sizeof(BatchItem) * items.size())) != PC_OK) return a;
        PC_CUDA(h, cudaMemcpy(dst, items.data(), sizeof(BatchItem) * items.size(), cudaMemcpyHostToDevice));
        h->q_nitems = (int)items.size();
        h->q_kind = item_kind(h->desc.dim, items.front().lft);
        (adj ? h->q_smem_b : h->q_smem) = smem;
    }
    if (!h->q_op_d && (a = dev_alloc(h, &h->q_op_d, sizeof(OpDev<float>))) != PC_OK) return a;
    if (!h->q_counter_d && (a = dev_alloc(h, &h->q_counter_d, sizeof(int))) != PC_OK) return a;
    PC_CUDA(h, cudaFuncSetAttribute(queue_kernel(h->q_kind), cudaFuncAttributeMaxDynamicSharedMemorySize, 110 * 1024));
    h->q_grid = persistent_grid(queue_kernel(h->q_kind), h->q_smem);
    return PC_OK;
}

// Enqueues one run of a batch on st: every operator's stage 0 and stage-1 sums (spread over
// the prep streams, so that the small launches of different operators overlap), the queue
// resets, the persistent kernels.
pc_status batch_enqueue(pc_batch* B, cudaStream_t st)
{
    const size_t np = B->prep.size();
    if (np && cudaEventRecord(B->prep_fork, st) != cudaSuccess) return PC_ERR_CUDA;
    for (size_t p = 0; p < np; ++p)
        if (cudaStreamWaitEvent(B->prep[p], B->prep_fork, 0) != cudaSuccess) return PC_ERR_CUDA;
    for (size_t i = 0; i < B->ops.size(); ++i) {
        pc_op* h = B->ops[i];
        cudaStream_t sp = np ? B->prep[i % np] : st;
        pc_status ps = prepare_t<float>(h, sp);
        if (ps == PC_OK) ps = s_rows_t<float>(h, B->od[i], sp, B->ops_d + i);
        if (ps != PC_OK) return ps;
    }
    for (size_t p = 0; p < np; ++p)
        if (cudaEventRecord(B->prep_join[p], B->prep[p]) != cudaSuccess ||
            cudaStreamWaitEvent(st, B->prep_join[p], 0) != cudaSuccess)
            return PC_ERR_CUDA;
    if (cudaMemsetAsync(B->counter_d, 0, sizeof(int) * B->groups.size(), st) != cudaSuccess) return PC_ERR_CUDA;
    const size_t ng = B->groups.size();
    if (ng > 1 && cudaEventRecord(B->fork[0], st) != cudaSuccess) return PC_ERR_CUDA;
    for (size_t gi = 0; gi < ng; ++gi) {
        const QGroup& q = B->groups[gi];
        cudaStream_t sg = gi ? B->side[gi - 1] : st;
        if (gi && cudaStreamWaitEvent(sg, B->fork[0], 0) != cudaSuccess) return PC_ERR_CUDA;
        queue_kernel(q.kind)<<<q.grid, 256, B->smem, sg>>>(B->ops_d, B->items_d + q.start, q.count,
                                                           B->counter_d + gi);
        count_launch();
        if (gi && (cudaEventRecord(B->join[gi - 1], sg) != cudaSuccess ||
                   cudaStreamWaitEvent(st, B->join[gi - 1], 0) != cudaSuccess))
            return PC_ERR_CUDA;
    }
    if (cudaGetLastError() != cudaSuccess) return PC_ERR_CUDA;
    for (pc_op* h : B->ops) {
        h->prepared = true;
        h->assembled = true;
        h->theta_gen++;
    }
    return PC_OK;
}

void batch_free(pc_batch* B)
{
    if (!B) return;
    if (B->exec) cudaGraphExecDestroy(B->exec);
    if (B->graph) cudaGraphDestroy(B->graph);
    if (B->cap) cudaStreamDestroy(B->cap);
    for (cudaStream_t s : B->side) cudaStreamDestroy(s);
    for (cudaStream_t s : B->prep) cudaStreamDestroy(s);
    for (cudaEvent_t e : B->prep_join) cudaEventDestroy(e);
    if (B->prep_fork) cudaEventDestroy(B->prep_fork);
    for (cudaEvent_t e : B->fork) cudaEventDestroy(e);
    for (cudaEvent_t e : B->join) cudaEventDestroy(e);
    if (B->ops_d) cudaFree(B->ops_d);
    if (B->items_d) cudaFree(B->items_d);
    if (B->counter_d) cudaFree(B->counter_d);
    delete B;
}

pc_status batch_build(pc_handle* ops, int count, cudaStream_t st, bool capture, pc_batch** out)
{
    *out = nullptr;
    if (!ops || count < 1) return fail(nullptr, PC_ERR_INVALID_ARG, "batch needs at least one operator");
    pc_batch* B = new (std::nothrow) pc_batch();
    if (!B) return fail(nullptr, PC_ERR_OOM, "host allocation failed");
    std::vector<OpDev<float>>& od = B->od;
    std::vector<ItemCand> cands;
    for (int i = 0; i < count; ++i) {
        pc_op* h = ops[i];
        if (!h) {
            batch_free(B);
            return fail(nullptr, PC_ERR_INVALID_ARG, "operator %d is NULL", i);
        }
        if (h->desc.precision != PC_FP32) {
            batch_free(B);
            return fail(nullptr, PC_ERR_UNSUPPORTED, "batches are FP32 only (operator %d is FP64)", i);
        }
        B->ops.push_back(h);
        od.push_back(make_opdev<float>(h));
        make_items(h, i, &cands, &B->smem);
    }
    // one range per kernel kind, longest items first within each
    std::stable_sort(cands.begin(), cands.end(), [](const ItemCand& a, const ItemCand& b) {
        const int ka = item_kind(a.it.dim, a.it.lft), kb = item_kind(b.it.dim, b.it.lft);
        return ka != kb ? ka < kb : a.cost > b.cost;
    });
    std::vector<BatchItem> items;
    for (const ItemCand& c : cands) {
        const int kind = item_kind(c.it.dim, c.it.lft);
        if (B->groups.empty() || B->groups.back().kind != kind)
            B->groups.push_back(QGroup{kind, (int)items.size(), 0, 0});
        B->groups.back().count++;
        items.push_back(c.it);
    }
    B->nitems = (int)items.size();
    cudaError_t e;
    if ((e = cudaMalloc(&B->ops_d, sizeof(OpDev<float>) * od.size())) ||
        (e = cudaMalloc(&B->items_d, sizeof(BatchItem) * items.size())) ||
        (e = cudaMalloc(&B->counter_d, sizeof(int) * B->groups.size())) ||
        (e = cudaMemcpyAsync(B->ops_d, od.data(), sizeof(OpDev<float>) * od.size(), cudaMemcpyHostToDevice, st)) ||
        (e = cudaMemcpyAsync(B->items_d, items.data(), sizeof(BatchItem) * items.size(), cudaMemcpyHostToDevice,
                             st))) {
        batch_free(B);
        return fail(nullptr, e == cudaErrorMemoryAllocation ? PC_ERR_OOM : PC_ERR_CUDA, "batch setup: %s",
                    cudaGetErrorString(e));
    }
    for (QGroup& q : B->groups) {
        if ((e = cudaFuncSetAttribute(queue_kernel(q.kind), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)B->smem)) != cudaSuccess) {
            batch_free(B);
            return fail(nullptr, PC_ERR_CUDA, "batch setup: %s", cudaGetErrorString(e));
        }
        q.grid = persistent_grid(queue_kernel(q.kind), B->smem);
    }
    B->kernels_per_run = 6 * count + (int)B->groups.size();
    for (pc_op* h : B->ops) B->kernels_per_run += (h->desc.dim == 2 && h->S_d) ? 1 : 0;  // k_s_tiles
    {
        cudaEvent_t ev;
        if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) {
            batch_free(B);
            return fail(nullptr, PC_ERR_CUDA, "batch setup: %s", cudaGetErrorString(e));
        }
        B->fork.push_back(ev);
        for (size_t gi = 1; gi < B->groups.size(); ++gi) {
            cudaStream_t s2;
            if ((e = cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking)) != cudaSuccess) {
                batch_free(B);
                return fail(nullptr, PC_ERR_CUDA, "batch setup: %s", cudaGetErrorString(e));
            }
            B->side.push_back(s2);
            if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) {
                batch_free(B);
                return fail(nullptr, PC_ERR_CUDA, "batch setup: %s", cudaGetErrorString(e));
            }
            B->join.push_back(ev);
        }
        if (count > 1) {
            if ((e = cudaEventCreateWithFlags(&B->prep_fork, cudaEventDisableTiming)) != cudaSuccess) {
                batch_free(B);
                return fail(nullptr, PC_ERR_CUDA, "batch setup: %s", cudaGetErrorString(e));
            }
            for (int p = 0; p < std::min(count, 8); ++p) {
                cudaStream_t s2;
                if ((e = cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking)) != cudaSuccess) {
                    batch_free(B);
                    return fail(nullptr, PC_ERR_CUDA, "batch setup: %s", cudaGetErrorString(e));
                }
                B->prep.push_back(s2);
                if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) {
                    batch_free(B);
                    return fail(nullptr, PC_ERR_CUDA, "batch setup: %s", cudaGetErrorString(e));
                }
                B->prep_join.push_back(ev);
            }
        }
    }
    // one eager run (sets up every kernel), then capture the same sequence
    pc_status ps = batch_enqueue(B, st);
    if (ps != PC_OK || (e = cudaStreamSynchronize(st)) != cudaSuccess) {
        batch_free(B);
        return fail(nullptr, PC_ERR_CUDA, "batch run failed");
    }
    if (capture) {
        if ((e = cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking)) ||
            (e = cudaStreamBeginCapture(B->cap, cudaStreamCaptureModeThreadLocal))) {
            batch_free(B);
            return fail(nullptr, PC_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
        }
        ps = batch_enqueue(B, B->cap);
        e = cudaStreamEndCapture(B->cap, &B->graph);
        if (ps != PC_OK || e != cudaSuccess || (e = cudaGraphInstantiate(&B->exec, B->graph, 0)) != cudaSuccess) {
            batch_free(B);
            return fail(nullptr, PC_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(e));
        }
    }
    *out = B;
    return PC_OK;
}

// Times one band's row-assembly launch (3 launches after a warm-up; minimum).
template <typename T>
float time_band(pc_op* h, const BandPlan& bp, cudaStream_t st)
{
    OpDev<T> od = make_opdev<T>(h);
    const int ctas = (bp.rows + bp.cfg.rpc - 1) / bp.cfg.rpc;
    const int threads = bp.cfg.gt * bp.cfg.rpc;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    float best = 1e30f;
    for (int it = 0; it < 4; ++it) {
        cudaEventRecord(a, st);
        if (h->desc.dim == 1)
            k_assemble1d<T><<<ctas, threads, bp.smem, st>>>(od, bp.cfg);
        else
            launch_asm2d<T>(h, od, bp, ctas, threads, st);
        cudaEventRecord(b, st);
        cudaEventSynchronize(b);
        float ms = 0;
        cudaEventElapsedTime(&ms, a, b);
        if (it > 0) best = std::min(best, ms);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return best;
}

template <typename T>
pc_status autotune_t(pc_op* h, cudaStream_t st)
{
    pc_status ps = prepare_t<T>(h, st);
    if (ps == PC_OK) ps = s_rows_t<T>(h, make_opdev<T>(h), st);  // the row kernels time on current s rows
    if (ps != PC_OK) return ps;
    h->prepared = true;
    if (h->desc.dim == 1 && set_smem_attr<T, 1>() != PC_OK) return fail(h, PC_ERR_CUDA, "cudaFuncSetAttribute failed");
    Geo g = geo_of(&h->desc);
    for (BandPlan& cur : h->plan) {
        BandPlan best = cur;
        float tbest = time_band<T>(h, cur, st);
        for (int gt : {32, 64, 128, 256}) {
            if (gt == cur.cfg.gt) continue;
            BandPlan cand;
            if (plan_band(h, g, cur.b, gt, &cand) != PC_OK) continue;
            const float t = time_band<T>(h, cand, st);
            if (t < tbest) {
                tbest = t;
                best = cand;
            }
        }
        cur = best;
    }
    PC_CUDA(h, cudaGetLastError());
    pc_status qs = build_queue(h);
    if (qs != PC_OK) return qs;
    // leave Theta assembled with the tuned plan
    return assemble_t<T>(h, st, 2);
}

}  // namespace

// =========================================================================================
// C-ABI
// =========================================================================================
// ---------------------------------------------------------------------------------------
// Wavelet-domain deblurring solver (Section 4.3; FISTA-W / FISTA-WP).  All of it runs on
// the stored Theta in its own precision (FP32 or FP64 values, never the BF16 copy).
// ---------------------------------------------------------------------------------------
namespace {

template <typename T>
pc_status solver_scratch(pc_op* h, T** y, T** r, T** g, double** nrm)
{
    const int64_t N = h->N;
    if (!h->fista_d) {
        char* p = nullptr;
        pc_status st = dev_alloc(h, &p, sizeof(T) * 3 * N + 2 * sizeof(double));
        if (st != PC_OK) return st;
        h->fista_d = p;
    }
    *y = (T*)h->fista_d;
    *r = *y + N;
    *g = *r + N;
    *nrm = (double*)(*g + N);
    return PC_OK;
}

inline int vec_blocks(int64_t N) { return (int)((N + 255) / 256); }

// r = Theta u, then g = Theta^T r (minus z0 in between when z0 is given)
template <typename T>
pc_status normal_apply(pc_op* h, const T* u, T* r, T* g, const T* z0, cudaStream_t st)
{
    // both products gather (the scattering one over the transposed copy)
    const T* vals = (const T*)h->theta_d;
    pc_status e = apply1_t<T, T, false>(h, vals, u, r, z0, false, st, true);
    if (e != PC_OK) return e;
    return apply1_t<T, T, false>(h, vals, r, g, nullptr, true, st, true);
}

template <typename T>
pc_status jacobi_t(pc_op* h, T* diag, cudaStream_t st)
{
    T *y, *r, *g;
    double* nrm;
    pc_status e = solver_scratch<T>(h, &y, &r, &g, &nrm);
    if (e != PC_OK) return e;
    k_fill_vec<T><<<vec_blocks(h->N), 256, 0, st>>>(y, h->N, T(1));
    count_launch();
    e = apply1_t<T, T, true>(h, (const T*)h->theta_d, y, diag, nullptr, true, st, true);
    if (e != PC_OK) return e;
    PC_CUDA(h, cudaGetLastError());
    return PC_OK;
}

template <typename T>
pc_status power_norm_t(pc_op* h, const T* sigma, int iters, double* out, cudaStream_t st)
{
    T *u, *r, *g;
    double* nrm;
    pc_status e = solver_scratch<T>(h, &u, &r, &g, &nrm);
    if (e != PC_OK) return e;
    const int64_t N = h->N;
    const int vb = vec_blocks(N);
    k_fill_vec<T><<<vb, 256, 0, st>>>(u, N, (T)(1.0 / std::sqrt((double)N)));
    count_launch();
    for (int it = 0; it < iters; ++it) {
        if (sigma) {
            k_scale_sqrt<T><<<vb, 256, 0, st>>>(u, sigma, N);
            count_launch();
        }
        if ((e = normal_apply<T>(h, u, r, g, nullptr, st)) != PC_OK) return e;
        if (sigma) {
            k_scale_sqrt<T><<<vb, 256, 0, st>>>(g, sigma, N);
            count_launch();
        }
        PC_CUDA(h, cudaMemsetAsync(nrm, 0, sizeof(double), st));
        k_norm2<T><<<std::min(vb, 1024), 256, 0, st>>>(g, N, nrm);
        k_normalize<T><<<vb, 256, 0, st>>>(u, g, N, nrm);
        count_launch(2);
    }
    double s2 = 0.0;
    PC_CUDA(h, cudaMemcpyAsync(&s2, nrm, sizeof(double), cudaMemcpyDeviceToHost, st));
    PC_CUDA(h, cudaStreamSynchronize(st));
    PC_CUDA(h, cudaGetLastError());
    *out = std::sqrt(s2);
    return PC_OK;
}

template <typename T>
pc_status fista_t(pc_op* h, const T* z0, const T* w, const T* sigma, T* z, int iters, double tau, cudaStream_t st)
{
    T *y, *r, *g;
    double* nrm;
    pc_status e = solver_scratch<T>(h, &y, &r, &g, &nrm);
    if (e != PC_OK) return e;
    const int64_t N = h->N;
    PC_CUDA(h, cudaMemcpyAsync(y, z, sizeof(T) * N, cudaMemcpyDeviceToDevice, st));
    for (int i = 1; i <= iters; ++i) {
        if ((e = normal_apply<T>(h, y, r, g, z0, st)) != PC_OK) return e;
        const T beta = (T)((double)(i - 1) / (double)(i + 2));
        k_fista_step<T><<<vec_blocks(N), 256, 0, st>>>(z, y, g, w, sigma, N, (T)tau, beta);
        count_launch();
    }
    PC_CUDA(h, cudaGetLastError());
    return PC_OK;
}

}  // namespace

extern "C" {

pc_status pc_plan_check(const pc_desc* desc) { return check_desc(desc, nullptr); }

pc_status pc_plan_nnz(const pc_desc* desc, int64_t* nnz)
{
    pc_status st = check_desc(desc, nullptr);
    if (st != PC_OK) return st;
    if (!nnz) return fail(nullptr, PC_ERR_INVALID_ARG, "nnz is NULL");
    Geo g = geo_of(desc);
    return plan_nnz(g, nullptr, nnz);
}

pc_status pc_plan_row(const pc_desc* desc, int64_t row, int64_t* cols, int64_t* count)
{
    pc_status st = check_desc(desc, nullptr);
    if (st != PC_OK) return st;
    if (!count) return fail(nullptr, PC_ERR_INVALID_ARG, "count is NULL");
    Geo g = geo_of(desc);
    int64_t N = (g.d == 2) ? (int64_t)g.n * g.n : g.n;
    if (row < 0 || row >= N) return fail(nullptr, PC_ERR_INVALID_ARG, "row out of range");
    int b, l0, l1;
    decode(g, row, &b, &l0, &l1);
    Band Bo = band_info(g.d, g.n, g.L, b);
    int64_t len = row_length(g, b, l0, l1);
    if (!cols) {
        *count = len;
        return PC_OK;
    }
    if (*count < len) return fail(nullptr, PC_ERR_INVALID_ARG, "cols holds %lld < %lld", (long long)*count, (long long)len);
    int64_t pos = 0;
    for (int b2 = 0; b2 < g.nb; ++b2) {
        if (!block_kept(g.d, g.n, g.L, g.gap, b, b2)) continue;
        Band B2 = band_info(g.d, g.n, g.L, b2);
        int f0 = 0, W0 = 1, f1, W1;
        stencil(Bo.j, Bo.e1, l1, B2.j, B2.e1, g.r, g.Lf, g.n, g.gap < 0, &f1, &W1);
        if (g.d == 2) stencil(Bo.j, Bo.e0, l0, B2.j, B2.e0, g.r, g.Lf, g.n, g.gap < 0, &f0, &W0);
        for (int a = 0; a < W0; ++a)
            for (int c = 0; c < W1; ++c)
                cols[pos++] = B2.off + (int64_t)pmod(f0 + a, B2.nj) * ((g.d == 2) ? B2.nj : 0) + pmod(f1 + c, B2.nj);
    }
    *count = len;
    return PC_OK;
}

pc_status pc_create(const pc_desc* desc, const void* u, const void* v, void* stream, pc_handle* out)
{
    if (!out) return fail(nullptr, PC_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    pc_status st = check_desc(desc, nullptr);
    if (st != PC_OK) return st;
    if (!u || !v) return fail(nullptr, PC_ERR_INVALID_ARG, "u and v must not be NULL");
    pc_op* h = new (std::nothrow) pc_op();
    if (!h) return fail(nullptr, PC_ERR_OOM, "host allocation failed");
    h->desc = *desc;
    const pc_desc& D = h->desc;
    Geo g = geo_of(desc);
    h->Lf = 2 * D.delta;
    h->K = 2 * D.radius + 1;
    h->Ku = (D.dim == 2) ? h->K * h->K : h->K;
    h->nb = g.nb;
    h->N = (D.dim == 2) ? (int64_t)D.n * D.n : D.n;
    h->esz = (D.precision == PC_FP64) ? 8 : 4;
    if (filter_taps(D.family, D.delta, h->h) != h->Lf) {
        delete h;
        return fail(nullptr, PC_ERR_INVALID_ARG, "filter taps failed for family=%d delta=%d", D.family, D.delta);
    }
    cudaStream_t s = (cudaStream_t)stream;
    auto bail = [&](pc_status e) {
        std::string msg = h->err;
        free_all(h);
        delete h;
        g_noh_error = msg;
        return e;
    };
    // pattern
    plan_nnz(g, &h->row_ptr_h, &h->nnz);
    if ((st = plan_bands(h)) != PC_OK) return bail(st);
    if (getenv("PCW_DEBUG"))
        for (const BandPlan& bp : h->plan)
            fprintf(stderr,
                    "band %2d rows %7d j[%d..%d] k0 %d gt %3d rpc %2d batch %3d arena %7d smem %7zu arena_b %7d "
                    "smem_b %7zu\n",
                    bp.b, bp.rows, bp.jlo, bp.jhi, bp.k0, bp.cfg.gt, bp.cfg.rpc, bp.cfg.batch, bp.cfg.arena, bp.smem,
                    bp.cfg_b.arena, bp.smem_b);
    // geometry of the base wavelets and filtered wavelets
    int acc = 0;
    for (int j = 1; j <= D.levels; ++j) {
        h->wofs[j] = acc;
        acc += 2 * wav_len(j, h->Lf);
    }
    h->wofs[D.levels + 1] = acc;
    h->wav_total = acc;
    FiltDev& fd = h->fd;
    fd.nb = h->nb;
    fd.d = D.dim;
    fd.n = D.n;
    fd.r = D.radius;
    fd.m = D.m;
    fd.Lf = h->Lf;
    fd.order = D.order;
    for (int i = 0; i < MAXL + 2; ++i) fd.wofs[i] = h->wofs[i];
    int64_t Fo = 0, Go = 0;
    for (int b = 0; b < h->nb; ++b) {
        Band B = band_info(D.dim, D.n, D.levels, b);
        FiltBand& fb = fd.band[b];
        fb.j = B.j;
        fb.e0 = B.e0;
        fb.e1 = B.e1;
        const int U = wav_len(B.j, h->Lf) + 2 * D.radius;
        fb.U1 = U;
        fb.U0 = (D.dim == 2) ? U : 1;
        fb.R1 = std::min(U, D.n);
        fb.R0 = (D.dim == 2) ? std::min(U, D.n) : 1;
        fb.Foff = Fo;
        fb.Goff = Go;
        // the window sums index a band's filtered wavelets with 32-bit offsets
        if ((int64_t)D.m * fb.R0 * fb.R1 >= ((int64_t)1 << 31))
            return bail(fail(h, PC_ERR_UNSUPPORTED, "band %d: %d terms x %d x %d region exceed 2^31 elements", b, D.m,
                             fb.R0, fb.R1));
        Fo += (int64_t)D.m * fb.R0 * fb.R1;
        Go += (int64_t)D.m * ((D.dim == 2) ? h->K : 1) * fb.U1;
    }
    h->Ftotal = Fo;
    h->Gtotal = Go;
    // per-band geometry of the backward phases 2 and 3
    {
        BwdDev& bd = h->bd;
        bd.n = D.n;
        bd.m = D.m;
        bd.nb = h->nb;
        bd.N = h->N;
        int64_t So = 0;
        for (int b = 0; b < h->nb; ++b) {
            Band B = band_info(D.dim, D.n, D.levels, b);
            BwdBand& bb = bd.band[b];
            bb.j = B.j;
            bb.nj = B.nj;
            bb.P0 = wav_off(B.j, B.e0, h->Lf) - D.radius;
            bb.P1 = wav_off(B.j, B.e1, h->Lf) - D.radius;
            bb.R0 = fd.band[b].R0;
            bb.R1 = fd.band[b].R1;
            bb.Foff = fd.band[b].Foff;
            bb.Soff = So;
            bb.rowoff = B.off;
            So += band_rows(g, b) * (int64_t)bb.R0 * bb.R1;
        }
        h->Stotal = So;
        bd.mp = (D.m + 3) / 4 * 4 + 4;  // the last float4 of a k-group may read 4 past m
        int64_t FTo = 0;
        for (int b = 0; b < h->nb; ++b) {
            bd.band[b].FToff = FTo;
            FTo += (int64_t)bd.band[b].R0 * bd.band[b].R1 * bd.mp;
        }
        h->FTtotal = (D.dim == 2 && D.precision == PC_FP32) ? FTo : 0;
    }
    // window tiles
    h->mwords = (D.m + 63) / 64;
    if (D.dim == 2) {
        h->ts0 = h->ts1 = std::min(16, D.n);
        h->tpa0 = h->tpa1 = D.n / h->ts1;
    } else {
        h->ts0 = 1;
        h->ts1 = std::min(256, D.n);
        h->tpa0 = 1;
        h->tpa1 = D.n / h->ts1;
    }
    // device buffers
    const size_t es = h->esz;
    if ((st = dev_alloc(h, &h->u_d, es * D.m * h->Ku)) || (st = dev_alloc(h, &h->v_d, es * D.m * h->N)) ||
        (st = dev_alloc(h, &h->taps64_d, sizeof(double) * h->Lf)) ||
        (st = dev_alloc(h, &h->wav64_d, sizeof(double) * h->wav_total)) ||
        (st = dev_alloc(h, &h->tapsT_d, es * 2 * h->Lf)) || (st = dev_alloc(h, &h->wavT_d, es * h->wav_total)) ||
        (st = dev_alloc(h, &h->F_d, es * h->Ftotal)) || (st = dev_alloc(h, &h->G_d, es * h->Gtotal)) ||
        (st = dev_alloc(h, &h->row_ptr_d, sizeof(int64_t) * (h->N + 1))) ||
        (st = dev_alloc(h, &h->theta_d, es * h->nnz)) ||
        (st = dev_alloc(h, &h->masks_d, sizeof(unsigned long long) * h->tpa0 * h->tpa1 * h->mwords)) ||
        (st = dev_alloc(h, &h->err_d, sizeof(int))))
        return bail(st);
    if (D.store_bf16 && (st = dev_alloc(h, &h->theta16_d, sizeof(__nv_bfloat16) * h->nnz))) return bail(st);
    if (D.store_bf16 && (st = dev_alloc(h, &h->xsplit_d, sizeof(unsigned) * 16 * h->N))) return bail(st);
    if (D.dim == 2) {
        // s scratch (stage 1 of the assembly, dL/ds of the backward) and the device copy of the
        // operator view that k_s_tiles reads
        if ((st = dev_alloc(h, &h->S_d, h->esz * h->Stotal)) ||
            (st = dev_alloc(h, &h->od_d, std::max(sizeof(OpDev<double>), sizeof(OpDev<float>)))))
            return bail(st);
    }
    cudaError_t e;
    if ((e = cudaMemcpyAsync(h->taps64_d, h->h, sizeof(double) * h->Lf, cudaMemcpyHostToDevice, s)) ||
        (e = cudaMemcpyAsync(h->row_ptr_d, h->row_ptr_h.data(), sizeof(int64_t) * (h->N + 1), cudaMemcpyHostToDevice,
                             s)) ||
        (e = cudaMemsetAsync(h->err_d, 0, sizeof(int), s)) ||
        (e = cudaMemcpyAsync(h->u_d, u, es * D.m * h->Ku, cudaMemcpyDefault, s)) ||
        (e = cudaMemcpyAsync(h->v_d, v, es * D.m * h->N, cudaMemcpyDefault, s)) || (e = cudaStreamSynchronize(s))) {
        fail(h, PC_ERR_CUDA, "upload failed: %s", cudaGetErrorString(e));
        return bail(PC_ERR_CUDA);
    }
    if ((st = build_window_list(h, s)) != PC_OK) return bail(st);
    if ((st = build_queue(h)) != PC_OK) return bail(st);
    *out = h;
    return PC_OK;
}

pc_status pc_set_params(pc_handle h, const void* u, const void* v, void* stream)
{
    if (!h) return fail(nullptr, PC_ERR_INVALID_ARG, "handle is NULL");
    const pc_desc& D = h->desc;
    cudaStream_t s = (cudaStream_t)stream;
    if (u) PC_CUDA(h, cudaMemcpyAsync(h->u_d, u, h->esz * D.m * h->Ku, cudaMemcpyDefault, s));
    if (v) PC_CUDA(h, cudaMemcpyAsync(h->v_d, v, h->esz * D.m * h->N, cudaMemcpyDefault, s));
    h->assembled = false;
    h->prepared = false;
    if (v) return build_window_list(h, s);
    return PC_OK;
}

void pc_destroy(pc_handle h)
{
    if (!h) return;
    cudaDeviceSynchronize();
    free_all(h);
    delete h;
}

pc_status pc_assemble(pc_handle h, void* stream)
{
    if (!h) return fail(nullptr, PC_ERR_INVALID_ARG, "handle is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    if (h->desc.precision == PC_FP64) return assemble_t<double>(h, s, 3);
    return assemble_t<float>(h, s, 3);
}

pc_status pc_assemble_stage(pc_handle h, int stage, void* stream)
{
    if (!h) return fail(nullptr, PC_ERR_INVALID_ARG, "handle is NULL");
    if (stage != 0 && stage != 1) return fail(h, PC_ERR_INVALID_ARG, "stage must be 0 or 1");
    cudaStream_t s = (cudaStream_t)stream;
    const int mask = stage == 0 ? 1 : 2;
    if (h->desc.precision == PC_FP64) return assemble_t<double>(h, s, mask);
    return assemble_t<float>(h, s, mask);
}

int64_t pc_launch_counter(void) { return (int64_t)g_launches.load(); }

pc_status pc_filter_taps(int family, int delta, double* h)
{
    if (!h) return fail(nullptr, PC_ERR_INVALID_ARG, "h is NULL");
    if (delta < 1 || delta > 10) return fail(nullptr, PC_ERR_INVALID_ARG, "delta must be in 1..10");
    if (family != PC_DAUBECHIES && family != PC_SYMMLET)
        return fail(nullptr, PC_ERR_INVALID_ARG, "family must be PC_DAUBECHIES or PC_SYMMLET (got %d)", family);
    if (filter_taps(family, delta, h) != 2 * delta)
        return fail(nullptr, PC_ERR_INVALID_ARG, "filter taps failed for family=%d delta=%d", family, delta);
    return PC_OK;
}

pc_status pc_apply(pc_handle h, const void* x, void* y, int nrhs, int ldx, int ldy, void* stream)
{
    if (!h) return fail(nullptr, PC_ERR_INVALID_ARG, "handle is NULL");
    if (!h->assembled) return fail(h, PC_ERR_NOT_ASSEMBLED, "pc_apply before pc_assemble");
    if (!x || !y || nrhs < 1 || nrhs > 64 || ldx < nrhs || ldy < nrhs)
        return fail(h, PC_ERR_INVALID_ARG, "bad x/y/nrhs/ldx/ldy (nrhs=%d ldx=%d ldy=%d)", nrhs, ldx, ldy);
    cudaStream_t s = (cudaStream_t)stream;
    if (h->desc.precision == PC_FP64)
        return apply_t<double, double>(h, (const double*)h->theta_d, (const double*)x, (double*)y, nrhs, ldx, ldy, s);
    if (h->theta16_d) return apply_t<__nv_bfloat16, float>(h, h->theta16_d, (const float*)x, (float*)y, nrhs, ldx, ldy, s);
    return apply_t<float, float>(h, (const float*)h->theta_d, (const float*)x, (float*)y, nrhs, ldx, ldy, s);
}

pc_status pc_apply_adjoint(pc_handle h, const void* x, void* y, int nrhs, int ldx, int ldy, void* stream)
{
    if (!h) return fail(nullptr, PC_ERR_INVALID_ARG, "handle is NULL");
    if (!h->assembled) return fail(h, PC_ERR_NOT_ASSEMBLED, "pc_apply_adjoint before pc_assemble");
    if (!x || !y || nrhs < 1 || nrhs > 64 || ldx < nrhs || ldy < nrhs)
        return fail(h, PC_ERR_INVALID_ARG, "bad x/y/nrhs/ldx/ldy (nrhs=%d ldx=%d ldy=%d)", nrhs, ldx, ldy);
    cudaStream_t s = (cudaStream_t)stream;
    if (h->desc.precision == PC_FP64)
        return apply_t<double, double>(h, (const double*)h->theta_d, (const double*)x, (double*)y, nrhs, ldx, ldy, s,
                                       true);
    if (h->theta16_d)
        return apply_t<__nv_bfloat16, float>(h, h->theta16_d, (const float*)x, (float*)y, nrhs, ldx, ldy, s, true);
    return apply_t<float, float>(h, (const float*)h->theta_d, (const float*)x, (float*)y, nrhs, ldx, ldy, s, true);
}

pc_status pc_jacobi(pc_handle h, void* diag, void* stream)
{
    if (!h) return fail(nullptr, PC_ERR_INVALID_ARG, "handle is NULL");
    if (!h->assembled) return fail(h, PC_ERR_NOT_ASSEMBLED, "pc_jacobi before pc_assemble");
    if (!diag) return fail(h, PC_ERR_INVALID_ARG, "diag must not be NULL");
    cudaStream_t s = (cudaStream_t)stream;
    if (h->desc.precision == PC_FP64) return jacobi_t<double>(h, (double*)diag, s);
    return jacobi_t<float>(h, (float*)diag, s);
}

pc_status pc_power_norm(pc_handle h, const void* sigma, int iters, double* norm2, void* stream)
{
    if (!h) return fail(nullptr, PC_ERR_INVALID_ARG, "handle is NULL");
    if (!h->assembled) return fail(h, PC_ERR_NOT_ASSEMBLED, "pc_power_norm before pc_assemble");
    if (!norm2 || iters < 1) return fail(h, PC_ERR_INVALID_ARG, "norm2 must not be NULL and iters >= 1");
    cudaStream_t s = (cudaStream_t)stream;
    if (h->desc.precision == PC_FP64) return power_norm_t<double>(h, (const double*)sigma, iters, norm2, s);
    return power_norm_t<float>(h, (const float*)sigma, iters, norm2, s);
}

pc_status pc_fista(pc_handle h, const void* z0, const void* w, const void* sigma, void* z, int iters, double tau,
                   void* stream)
{
    if (!h) return fail(nullptr, PC_ERR_INVALID_ARG, "handle is NULL");
    if (!h->assembled) return fail(h, PC_ERR_NOT_ASSEMBLED, "pc_fista before pc_assemble");
    if (!z0 || !w || !z || iters < 0 || !(tau > 0.0))
        return fail(h, PC_ERR_INVALID_ARG, "bad z0/w/z/iters/tau (iters=%d tau=%g)", iters, tau);
    cudaStream_t s = (cudaStream_t)stream;
    if (h->desc.precision == PC_FP64)
        return fista_t<double>(h, (const double*)z0, (const double*)w, (const double*)sigma, (double*)z, iters, tau,
                               s);
    return fista_t<float>(h, (const float*)z0, (const float*)w, (const float*)sigma, (float*)z, iters, tau, s);
}

pc_status pc_backward(pc_handle h, const void* dtheta, void* du, void* dv, void* stream)
{
    if (!h) return fail(nullptr, PC_ERR_INVALID_ARG, "handle is NULL");
    if (!dtheta || !du || !dv) return fail(h, PC_ERR_INVALID_ARG, "dtheta, du and dv must not be NULL");
    cudaStream_t s = (cudaStream_t)stream;
    if (h->desc.precision == PC_FP64) return backward_t<double>(h, (const double*)dtheta, (double*)du, (double*)dv, s);
    return backward_t<float>(h, (const float*)dtheta, (float*)du, (float*)dv, s);
}

pc_status pc_backward_noalloc(pc_handle h, const void* dtheta, void* du, void* dv, void* stream)
{
    if (!h) return fail(nullptr, PC_ERR_INVALID_ARG, "handle is NULL");
    if (!dtheta || !du || !dv) return fail(h, PC_ERR_INVALID_ARG, "dtheta, du and dv must not be NULL");
    cudaStream_t s = (cudaStream_t)stream;
    if (h->desc.precision == PC_FP64)
        return backward_noalloc_t<double>(h, (const double*)dtheta, (double*)du, (double*)dv, s);
    return backward_noalloc_t<float>(h, (const float*)dtheta, (float*)du, (float*)dv, s);
}

pc_status pc_batch_create(pc_handle* ops, int count, void* stream, pc_batch_handle* out)
{
    if (!out) return fail(nullptr, PC_ERR_INVALID_ARG, "out is NULL");
    return batch_build(ops, count, (cudaStream_t)stream, true, out);
}

pc_status pc_batch_run(pc_batch_handle b, void* stream)
{
    if (!b || !b->exec) return fail(nullptr, PC_ERR_INVALID_ARG, "batch is NULL or not captured");
    // descriptors may have changed (window lists are rebuilt by pc_set_params): refresh them
    for (size_t i = 0; i < b->ops.size(); ++i) b->od[i] = make_opdev<float>(b->ops[i]);
    cudaError_t e = cudaMemcpyAsync(b->ops_d, b->od.data(), sizeof(OpDev<float>) * b->od.size(),
                                    cudaMemcpyHostToDevice, (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaGraphLaunch(b->exec, (cudaStream_t)stream);
    if (e != cudaSuccess) return fail(nullptr, PC_ERR_CUDA, "cudaGraphLaunch: %s", cudaGetErrorString(e));
    count_launch(b->kernels_per_run);
    for (pc_op* h : b->ops) {
        h->prepared = true;
        h->assembled = true;
        h->theta_gen++;
    }
    return PC_OK;
}

pc_status pc_batch_info(pc_batch_handle b, int* items, int* kernels_per_run)
{
    if (!b) return fail(nullptr, PC_ERR_INVALID_ARG, "batch is NULL");
    if (items) *items = b->nitems;
    if (kernels_per_run) *kernels_per_run = b->kernels_per_run;
    return PC_OK;
}

void pc_batch_destroy(pc_batch_handle b)
{
    if (!b) return;
    cudaDeviceSynchronize();
    batch_free(b);
}

pc_status pc_batch_assemble(pc_handle* ops, int count, void* stream)
{
    pc_batch* B = nullptr;
    pc_status st = batch_build(ops, count, (cudaStream_t)stream, false, &B);
    if (st != PC_OK) return st;
    batch_free(B);  // the eager run in batch_build assembled every operator (synchronised)
    return PC_OK;
}

pc_status pc_autotune(pc_handle h, void* stream)
{
    if (!h) return fail(nullptr, PC_ERR_INVALID_ARG, "handle is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    if (h->desc.precision == PC_FP64) return autotune_t<double>(h, s);
    return autotune_t<float>(h, s);
}

pc_status pc_info(pc_handle h, int64_t* nnz, int64_t* device_bytes)
{
    if (!h) return fail(nullptr, PC_ERR_INVALID_ARG, "handle is NULL");
    if (nnz) *nnz = h->nnz;
    if (device_bytes) *device_bytes = h->dev_bytes;
    return PC_OK;
}

pc_status pc_theta(pc_handle h, void** values, void** values_bf16, int64_t** row_ptr)
{
    if (!h) return fail(nullptr, PC_ERR_INVALID_ARG, "handle is NULL");
    if (values) *values = h->theta_d;
    if (values_bf16) *values_bf16 = h->theta16_d;
    if (row_ptr) *row_ptr = h->row_ptr_d;
    return PC_OK;
}

pc_status pc_lookup(pc_handle h, int64_t n, const int64_t* mu, const int64_t* lambda, int64_t* pos)
{
    if (!h) return fail(nullptr, PC_ERR_INVALID_ARG, "handle is NULL");
    if (n < 0 || (n > 0 && (!mu || !lambda || !pos))) return fail(h, PC_ERR_INVALID_ARG, "bad arrays");
    Geo g = geo_of(&h->desc);
    for (int64_t i = 0; i < n; ++i) {
        int64_t s = mu[i], c = lambda[i];
        if (h->desc.order == PC_ORDER_CONV_THEN_MULT) std::swap(s, c);
        pos[i] = -1;
        if (s < 0 || s >= h->N || c < 0 || c >= h->N) continue;
        int b, l0, l1, b2, m0, m1;
        decode(g, s, &b, &l0, &l1);
        decode(g, c, &b2, &m0, &m1);
        if (!block_kept(g.d, g.n, g.L, g.gap, b, b2)) continue;
        Band Bo = band_info(g.d, g.n, g.L, b), B2 = band_info(g.d, g.n, g.L, b2);
        int f0 = 0, W0 = 1, f1, W1;
        stencil(Bo.j, Bo.e1, l1, B2.j, B2.e1, g.r, g.Lf, g.n, g.gap < 0, &f1, &W1);
        if (g.d == 2) stencil(Bo.j, Bo.e0, l0, B2.j, B2.e0, g.r, g.Lf, g.n, g.gap < 0, &f0, &W0);
        const int a = (g.d == 2) ? pmod(m0 - f0, B2.nj) : 0, bb = pmod(m1 - f1, B2.nj);
        if (a >= W0 || bb >= W1) continue;
        int64_t off = 0;
        for (int q = 0; q < b2; ++q)
            if (block_kept(g.d, g.n, g.L, g.gap, b, q)) off += block_count(g.d, g.n, g.L, g.Lf, g.r, g.gap, b, l0, l1, q);
        pos[i] = h->row_ptr_h[s] + off + (int64_t)a * W1 + bb;
    }
    return PC_OK;
}

pc_status pc_export(pc_handle h, int64_t* row_ptr, int64_t* cols, double* vals, void* stream)
{
    if (!h) return fail(nullptr, PC_ERR_INVALID_ARG, "handle is NULL");
    if (!h->assembled) return fail(h, PC_ERR_NOT_ASSEMBLED, "pc_export before pc_assemble");
    if (!row_ptr || !cols || !vals) return fail(h, PC_ERR_INVALID_ARG, "row_ptr, cols and vals must not be NULL");
    const int64_t N = h->N, nnz = h->nnz;
    // stored values to the host, as double
    std::vector<double> sv((size_t)nnz);
    if (h->desc.precision == PC_FP64) {
        PC_CUDA(h, cudaMemcpyAsync(sv.data(), h->theta_d, sizeof(double) * nnz, cudaMemcpyDeviceToHost,
                                   (cudaStream_t)stream));
        PC_CUDA(h, cudaStreamSynchronize((cudaStream_t)stream));
    } else {
        std::vector<float> f((size_t)nnz);
        PC_CUDA(h, cudaMemcpyAsync(f.data(), h->theta_d, sizeof(float) * nnz, cudaMemcpyDeviceToHost,
                                   (cudaStream_t)stream));
        PC_CUDA(h, cudaStreamSynchronize((cudaStream_t)stream));
        for (int64_t i = 0; i < nnz; ++i) sv[(size_t)i] = f[(size_t)i];
    }
    // the pattern is symmetric, so row mu of Theta has as many entries as stored row mu
    for (int64_t i = 0; i <= N; ++i) row_ptr[i] = h->row_ptr_h[(size_t)i];
    Geo g = geo_of(&h->desc);
    const bool conv_first = h->desc.order == PC_ORDER_CONV_THEN_MULT;   // stored row = column of Theta
    std::vector<int64_t> cursor;
    if (conv_first) cursor.assign(h->row_ptr_h.begin(), h->row_ptr_h.end() - 1);
    std::vector<std::pair<int64_t, double>> row;
    for (int64_t s = 0; s < N; ++s) {
        int b, l0, l1;
        decode(g, s, &b, &l0, &l1);
        const Band Bo = band_info(g.d, g.n, g.L, b);
        int64_t pos = h->row_ptr_h[(size_t)s];
        row.clear();
        for (int b2 = 0; b2 < g.nb; ++b2) {
            if (!block_kept(g.d, g.n, g.L, g.gap, b, b2)) continue;
            const Band B2 = band_info(g.d, g.n, g.L, b2);
            int f0 = 0, W0 = 1, f1, W1;
            stencil(Bo.j, Bo.e1, l1, B2.j, B2.e1, g.r, g.Lf, g.n, g.gap < 0, &f1, &W1);
            if (g.d == 2) stencil(Bo.j, Bo.e0, l0, B2.j, B2.e0, g.r, g.Lf, g.n, g.gap < 0, &f0, &W0);
            for (int a = 0; a < W0; ++a)
                for (int c = 0; c < W1; ++c) {
                    const int64_t col =
                        B2.off + (int64_t)pmod(f0 + a, B2.nj) * ((g.d == 2) ? B2.nj : 0) + pmod(f1 + c, B2.nj);
                    row.emplace_back(col, sv[(size_t)pos++]);
                }
        }
        if (pos != h->row_ptr_h[(size_t)s + 1]) return fail(h, PC_ERR_DEVICE, "internal: row %lld length", (long long)s);
        if (!conv_first) {
            // Theta's row s: sort by column
            std::sort(row.begin(), row.end(),
                      [](const std::pair<int64_t, double>& x, const std::pair<int64_t, double>& y) {
                          return x.first < y.first;
                      });
            int64_t o = h->row_ptr_h[(size_t)s];
            for (const auto& e : row) {
                cols[o] = e.first;
                vals[o++] = e.second;
            }
        } else {
            // Theta[col, s]: appended to row col; s ascends, so every row ends up sorted
            for (const auto& e : row) {
                const int64_t o = cursor[(size_t)e.first]++;
                if (o >= h->row_ptr_h[(size_t)e.first + 1])
                    return fail(h, PC_ERR_DEVICE, "internal: pattern not symmetric at row %lld", (long long)e.first);
                cols[o] = s;
                vals[o] = e.second;
            }
        }
    }
    return PC_OK;
}

pc_status pc_sync(pc_handle h, void* stream)
{
    if (!h) return fail(nullptr, PC_ERR_INVALID_ARG, "handle is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    PC_CUDA(h, cudaStreamSynchronize(s));
    int flag = 0;
    PC_CUDA(h, cudaMemcpy(&flag, h->err_d, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) {
        PC_CUDA(h, cudaMemset(h->err_d, 0, sizeof(int)));
        return fail(h, PC_ERR_DEVICE, "device fault flag 0x%x (1: arena overflow, 2: row length, 4: index, 8: queue)",
                    flag);
    }
    return PC_OK;
}

const char* pc_last_error(pc_handle h) { return h ? h->err.c_str() : g_noh_error.c_str(); }

pc_status pc_svir_expansion(const float* S, int64_t N, int K, int m, int l, int power_iters, const float* omega,
                            float* u, float* v, double* sing, void* stream)
{
    if (!S || !omega || !u || !v || N < 1 || K < 1 || m < 1 || l < m || l > 64 || l > K || power_iters < 0 ||
        N > ((int64_t)1 << 30))
        return fail(nullptr, PC_ERR_INVALID_ARG, "pc_svir_expansion: bad arguments (need 1 <= m <= l <= min(64, K))");
    SvirWork w;
    w.st = (cudaStream_t)stream;
    float *Y = nullptr, *Z = nullptr, *Bm = nullptr, *Ut = nullptr;
    auto cleanup = [&]() {
        for (void* p : {(void*)Y, (void*)Z, (void*)Bm, (void*)Ut, (void*)w.G, (void*)w.T, (void*)w.tmp})
            if (p) cudaFree(p);
        if (w.hb) cublasDestroy(w.hb);
    };
    auto bad = [&](pc_status st, const std::string& msg) {
        cleanup();
        return fail(nullptr, st, "pc_svir_expansion: %s", msg.c_str());
    };
    const int64_t rows = std::max<int64_t>(N, K);
    if (cudaMalloc(&Y, sizeof(float) * N * l) || cudaMalloc(&Z, sizeof(float) * (size_t)K * l) ||
        cudaMalloc(&Bm, sizeof(float) * (size_t)l * K) || cudaMalloc(&Ut, sizeof(float) * (size_t)m * l) ||
        cudaMalloc(&w.G, sizeof(float) * l * l) || cudaMalloc(&w.T, sizeof(float) * l * l) ||
        cudaMalloc(&w.tmp, sizeof(float) * rows * l))
        return bad(PC_ERR_OOM, "device allocation failed");
    if (cublasCreate(&w.hb) != CUBLAS_STATUS_SUCCESS || cublasSetStream(w.hb, w.st) != CUBLAS_STATUS_SUCCESS ||
        cublasSetMathMode(w.hb, CUBLAS_PEDANTIC_MATH) != CUBLAS_STATUS_SUCCESS)
        return bad(PC_ERR_CUDA, "cuBLAS set-up failed");
    // range finder: Y = S Omega, orthonormalised; power iterations Z = S^T Q, Y = S Z
    if (gemm_rm(w.hb, false, false, (int)N, l, K, S, K, omega, l, Y, l) != CUBLAS_STATUS_SUCCESS)
        return bad(PC_ERR_CUDA, "cuBLAS product S Omega failed");
    int r = svir_orthonormalise(w, Y, N, l, l);
    if (!r) return bad(PC_ERR_CUDA, w.err);
    for (int it = 0; it < power_iters; ++it) {
        if (gemm_rm(w.hb, true, false, K, r, (int)N, S, K, Y, l, Z, l) != CUBLAS_STATUS_SUCCESS)
            return bad(PC_ERR_CUDA, "cuBLAS product S^T Q failed");
        int rz = svir_orthonormalise(w, Z, K, r, l);
        if (!rz) return bad(PC_ERR_CUDA, w.err);
        if (gemm_rm(w.hb, false, false, (int)N, rz, K, S, K, Z, l, Y, l) != CUBLAS_STATUS_SUCCESS)
            return bad(PC_ERR_CUDA, "cuBLAS product S Z failed");
        r = svir_orthonormalise(w, Y, N, rz, l);
        if (!r) return bad(PC_ERR_CUDA, w.err);
    }
    // projected matrix B = Q^T S (r x K), its SVD on the host in FP64
    if (gemm_rm(w.hb, true, false, r, K, (int)N, Y, l, S, K, Bm, K) != CUBLAS_STATUS_SUCCESS)
        return bad(PC_ERR_CUDA, "cuBLAS product Q^T S failed");
    std::vector<float> bf((size_t)r * K);
    if (cudaMemcpyAsync(bf.data(), Bm, sizeof(float) * bf.size(), cudaMemcpyDeviceToHost, w.st) != cudaSuccess ||
        cudaStreamSynchronize(w.st) != cudaSuccess)
        return bad(PC_ERR_CUDA, "copy of the projected matrix failed");
    std::vector<double> B(bf.begin(), bf.end()), sv, U, W;
    jacobi_svd(B, r, K, &sv, &U, &W);
    // u_k = W[:, k]; v_k = s_k (Q U)[:, k], as v (m x N) = (U[:, :m] diag(s))^T Q^T; terms past the
    // numerical rank of the sketch are zero
    const int mm = std::min(m, r);
    std::vector<float> uh((size_t)m * K, 0.0f), ut((size_t)m * l, 0.0f);
    for (int k = 0; k < mm; ++k) {
        for (int t = 0; t < K; ++t) uh[(size_t)k * K + t] = (float)W[(size_t)t * r + k];
        for (int j = 0; j < r; ++j) ut[(size_t)k * l + j] = (float)(U[(size_t)j * r + k] * sv[k]);
    }
    if (cudaMemcpyAsync(u, uh.data(), sizeof(float) * uh.size(), cudaMemcpyHostToDevice, w.st) != cudaSuccess ||
        cudaMemcpyAsync(Ut, ut.data(), sizeof(float) * ut.size(), cudaMemcpyHostToDevice, w.st) != cudaSuccess)
        return bad(PC_ERR_CUDA, "copy of the factors failed");
    if (gemm_rm(w.hb, false, true, m, (int)N, r, Ut, l, Y, l, v, (int)N) != CUBLAS_STATUS_SUCCESS)
        return bad(PC_ERR_CUDA, "cuBLAS product for v failed");
    if (cudaStreamSynchronize(w.st) != cudaSuccess) return bad(PC_ERR_CUDA, "stream synchronisation failed");
    if (sing)
        for (int i = 0; i < l; ++i) sing[i] = i < r ? sv[i] : 0.0;
    cleanup();
    return PC_OK;
}

}  // extern "C"

// =========================================================================================
// Thresholded Algorithm 1 (Section 3.2): Theta~ = sum_k A~_k B_k, see pcw_alg1.cuh
// =========================================================================================
struct pc_alg1 {
    int D = 1, n = 0, J = 0, Lf = 0, m = 0, r = 0, ncls = 0, nJ = 0, rows = 0;
    int64_t N = 0, nnz = 0;
    double eta = 0.0;
    std::vector<pcw::alg1::A1Class> cls;
    std::vector<int> band_cbase;  // first class of each canonical band
    std::vector<double> tau;
    std::vector<int64_t> kept;
    double stage_ms[4] = {0, 0, 0, 0};
    bool fp32 = false;            // Theta~ in FP32 (products in FP32), else FP64
    bool discard = false;         // rows formed into one reused buffer, Theta~ not kept
    int rule = PC_ALG1_SCHUR;     // threshold rule
    void* theta_d = nullptr;
    std::string err = "no error";
};

namespace {

using pcw::alg1::A1Class;
using pcw::alg1::A1Params;
using pcw::alg1::Ax;

// Canonical band b of a basis with levels J: level, types (e0, e1) and the offset of its first
// coefficient.  Band 0 is the approximation of level J; then levels J..1, in 2-D the detail
// bands (0,1), (1,0), (1,1).
struct BandId {
    int j, e0, e1;
    int64_t off;
};

std::vector<BandId> canonical_bands(int D, int n, int J)
{
    std::vector<BandId> out;
    const int64_t nJ = n >> J;
    out.push_back({J, 0, 0, 0});
    for (int l = J; l >= 1; --l) {
        const int64_t nl = n >> l;
        if (D == 2) {
            out.push_back({l, 0, 1, nl * nl});
            out.push_back({l, 1, 0, 2 * nl * nl});
            out.push_back({l, 1, 1, 3 * nl * nl});
        } else {
            out.push_back({l, 1, 0, nl});
        }
    }
    (void)nJ;
    return out;
}

// Calls f(band index, level, e0, e1, offset in the row, box0, box1) for the segments of a row.
template <class Fn>
void host_segments(int D, int J, const Ax (*bx)[pcw::alg1::A1_MAXJ + 1], const int* offl, Fn f)
{
    f(0, J, 0, 0, 0, bx[0][J], bx[1][J]);
    int band = 1;
    for (int l = J; l >= 1; --l) {
        const int sz = bx[0][l].w * bx[1][l].w;
        if (D == 2) {
            f(band++, l, 0, 1, offl[l], bx[0][l], bx[1][l]);
            f(band++, l, 1, 0, offl[l] + sz, bx[0][l], bx[1][l]);
            f(band++, l, 1, 1, offl[l] + 2 * sz, bx[0][l], bx[1][l]);
        } else {
            f(band++, l, 1, 0, offl[l], bx[0][l], bx[1][l]);
        }
    }
}

// Temporary device buffers of one call, stream-ordered on the call's stream (the pool allocator:
// no device-wide synchronisation per allocation), freed in stream order on exit.
struct DevBufs {
    cudaStream_t st;
    std::vector<void*> ptrs;
    explicit DevBufs(cudaStream_t s) : st(s) {}
    ~DevBufs()
    {
        for (void* p : ptrs)
            if (p) cudaFreeAsync(p, st);
    }
    template <class T>
    bool alloc(T** p, size_t count)
    {
        *p = nullptr;
        if (cudaMallocAsync((void**)p, sizeof(T) * std::max<size_t>(count, 1), st) != cudaSuccess) {
            *p = nullptr;
            (void)cudaGetLastError();  // an allocation failure is reported by status, not left pending
            return false;
        }
        ptrs.push_back(*p);
        return true;
    }
};

// Launch shape of a CTA-per-item kernel with `per_cta` doubles of scratch: dynamic shared memory
// when it fits (grid from the occupancy), else one global slab per CTA (grid of 2 per SM).
struct ScratchPlan {
    bool smem = true;
    int grid = 1;
    size_t bytes = 0;
};

template <class K>
ScratchPlan plan_scratch(K kernel, long long items, size_t per_cta, size_t elem = sizeof(double))
{
    ScratchPlan sp;
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    sp.bytes = per_cta * elem;
    if (sp.bytes <= 200 * 1024) {
        cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sp.bytes);
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, pcw::alg1::A1_THREADS, sp.bytes);
        sp.grid = (int)std::min<long long>(items, (long long)std::max(per_sm, 1) * sms);
    } else {
        sp.smem = false;
        sp.grid = (int)std::min<long long>(items, 2LL * sms);
    }
    sp.grid = std::max(sp.grid, 1);
    return sp;
}

pc_status a1_fail(pc_alg1* h, pc_status st, const std::string& msg)
{
    if (h) h->err = msg;
    return fail(nullptr, st, "pc_alg1_create: %s", msg.c_str());
}

template <int D>
pc_status alg1_run(pc_alg1* h, const pc_desc* desc, const double* u, const double* v, cudaStream_t st)
{
    using namespace pcw::alg1;
    const int n = h->n, J = h->J, Lf = h->Lf, m = h->m, r = h->r, ncls = h->ncls;
    const int64_t N = h->N;
    DevBufs db(st);
    auto oom = [&]() { return a1_fail(h, PC_ERR_OOM, "device allocation failed"); };
    auto cuda_err = [&](const char* what) { return a1_fail(h, PC_ERR_CUDA, std::string(what) + " failed"); };

    // taps and 1-D factor tables
    A1Params P{};
    P.D = D;
    P.n = n;
    P.J = J;
    P.Lf = Lf;
    P.r = r;
    P.m = m;
    P.ncls = ncls;
    P.nJ = h->nJ;
    P.N = N;
    double hh[64];
    if (pcw::filter_taps(desc->family, desc->delta, hh) != Lf) return a1_fail(h, PC_ERR_INVALID_ARG, "filter taps");
    for (int i = 0; i < Lf; ++i) P.h[i] = hh[i];
    for (int i = 2 - Lf; i <= 1; ++i) P.g[i - (2 - Lf)] = (((1 - i) % 2 == 0) ? 1.0 : -1.0) * hh[1 - i];
    for (int i = 0; i < Lf; ++i) {
        P.hf[i] = (float)P.h[i];
        P.gf[i] = (float)P.g[i];
    }
    std::vector<std::vector<double>> phi, psi;
    factor_tables(hh, Lf, J, &phi, &psi);
    std::vector<double> tab;
    for (int j = 1; j <= J; ++j) {
        P.tab_len[j] = (int)phi[j].size();
        P.tab_off[j][0] = (int)tab.size();
        tab.insert(tab.end(), phi[j].begin(), phi[j].end());
        P.tab_off[j][1] = (int)tab.size();
        tab.insert(tab.end(), psi[j].begin(), psi[j].end());
    }

    // classes with their generator boxes (the support of F widened by r), in canonical band order
    const std::vector<BandId> bands = canonical_bands(D, n, J);
    h->band_cbase.clear();
    h->cls.clear();
    int64_t gtotal = 0;
    for (const BandId& b : bands) {
        h->band_cbase.push_back((int)h->cls.size());
        const int ph = 1 << (J - b.j);
        for (int p0 = 0; p0 < ph; ++p0)
            for (int p1 = 0; p1 < (D == 2 ? ph : 1); ++p1) {
                A1Class c{};
                c.j = b.j;
                c.e0 = b.e0;
                c.e1 = (D == 2) ? b.e1 : 0;
                c.p0 = p0;
                c.p1 = p1;
                c.rows = h->rows;
                const int len = ((1 << b.j) - 1) * (Lf - 1) + 1;
                Ax b0[2];
                const int ee[2] = {c.e0, c.e1}, pp[2] = {p0, p1};
                for (int d = 0; d < 2; ++d) {
                    if (d >= D) {
                        b0[d] = {0, 1};
                        continue;
                    }
                    const int s = factor_start(b.j, ee[d], pp[d], Lf);
                    b0[d] = (len + 2 * r >= n) ? Ax{0, n} : Ax{s - r, len + 2 * r};
                }
                c.glen = chain(D, n, J, Lf, b0, c.g, c.goffl);
                c.goff = gtotal;
                gtotal += c.glen;
                h->cls.push_back(c);
            }
    }
    h->band_cbase.push_back((int)h->cls.size());
    if ((int)h->cls.size() != ncls) return a1_fail(h, PC_ERR_INVALID_ARG, "class count");
    P.gtotal = gtotal;

    // segments: the entries of each row class grouped by column class (class of the entry's
    // position: band, y mod 2^(J - l) per axis), and the segments of each column class
    std::vector<int> perm, seg_len, seg_row_off(ncls + 1, 0), seg_cc;
    std::vector<long long> seg_start;
    if (h->rule == PC_ALG1_SCHUR) {
        // (the plain cut needs no sums) a stable counting sort of each row's entries by column
        // class, over the few column classes the row meets
        perm.resize((size_t)gtotal);
        std::vector<int> cnt(ncls, 0), keys, ccs;
        for (int c = 0; c < ncls; ++c) {
            const A1Class& C = h->cls[c];
            ccs.assign((size_t)C.glen, 0);
            keys.clear();
            host_segments(D, J, C.g, C.goffl, [&](int band, int l, int, int, int off, Ax b0, Ax b1) {
                const int ph = 1 << (J - l);
                for (int i0 = 0; i0 < b0.w; ++i0)
                    for (int i1 = 0; i1 < b1.w; ++i1) {
                        const int q0 = (b0.a + i0) & (ph - 1), q1 = (D == 2) ? ((b1.a + i1) & (ph - 1)) : 0;
                        const int cc = h->band_cbase[band] + (D == 2 ? q0 * ph + q1 : q0);
                        if (cnt[cc]++ == 0) keys.push_back(cc);
                        ccs[(size_t)off + i0 * b1.w + i1] = cc;
                    }
            });
            std::sort(keys.begin(), keys.end());
            seg_row_off[c] = (int)seg_len.size();
            long long pos = C.goff;
            for (int cc : keys) {  // segment start of each key, then the count is reused as a cursor
                seg_cc.push_back(cc);
                seg_start.push_back(pos);
                seg_len.push_back(cnt[cc]);
                const long long st0 = pos;
                pos += cnt[cc];
                cnt[cc] = (int)(st0 - C.goff);
            }
            for (int e = 0; e < C.glen; ++e) perm[(size_t)C.goff + cnt[ccs[(size_t)e]]++] = e;
            for (int cc : keys) cnt[cc] = 0;
        }
    }
    const int nseg = (int)seg_len.size();
    seg_row_off[ncls] = nseg;

    std::vector<int> colseg_off(ncls + 1, 0), colseg(nseg);
    for (int s = 0; s < nseg; ++s) colseg_off[seg_cc[s] + 1]++;
    for (int c = 0; c < ncls; ++c) colseg_off[c + 1] += colseg_off[c];
    {
        std::vector<int> fill(colseg_off.begin(), colseg_off.end() - 1);
        for (int s = 0; s < nseg; ++s) colseg[fill[seg_cc[s]]++] = s;
    }

    // device buffers
    double *tab_d, *u_d, *v_d, *G_d, *segsum_d, *st_d, *vmax_d, *amax_d;
    A1Class* cls_d;
    int *perm_d, *seglen_d, *segrow_d, *colo_d, *cols_d, *done_d, *rbox_d;
    long long *segst_d, *kept_d;
    const int K = (D == 2) ? (2 * r + 1) * (2 * r + 1) : 2 * r + 1;
    if (!db.alloc(&tab_d, tab.size()) || !db.alloc(&cls_d, ncls) || !db.alloc(&u_d, (size_t)m * K) ||
        !db.alloc(&v_d, (size_t)m * N) || !db.alloc(&G_d, (size_t)m * gtotal) || !db.alloc(&perm_d, perm.size()) ||
        !db.alloc(&seglen_d, nseg) || !db.alloc(&segrow_d, ncls + 1) || !db.alloc(&colo_d, ncls + 1) ||
        !db.alloc(&cols_d, nseg) || !db.alloc(&segst_d, nseg) || !db.alloc(&segsum_d, (size_t)m * nseg) ||
        !db.alloc(&st_d, 6 * (size_t)m) || !db.alloc(&done_d, m) || !db.alloc(&vmax_d, m) || !db.alloc(&amax_d, m) ||
        !db.alloc(&kept_d, (size_t)m * ncls) || !db.alloc(&rbox_d, 4 * (size_t)ncls))
        return oom();
    if (cudaMemcpyAsync(tab_d, tab.data(), sizeof(double) * tab.size(), cudaMemcpyHostToDevice, st) ||
        cudaMemcpyAsync(cls_d, h->cls.data(), sizeof(A1Class) * ncls, cudaMemcpyHostToDevice, st) ||
        cudaMemcpyAsync(u_d, u, sizeof(double) * m * K, cudaMemcpyDefault, st) ||
        cudaMemcpyAsync(v_d, v, sizeof(double) * m * N, cudaMemcpyDefault, st) ||
        (nseg && (cudaMemcpyAsync(perm_d, perm.data(), sizeof(int) * perm.size(), cudaMemcpyHostToDevice, st) ||
                  cudaMemcpyAsync(seglen_d, seg_len.data(), sizeof(int) * nseg, cudaMemcpyHostToDevice, st) ||
                  cudaMemcpyAsync(segrow_d, seg_row_off.data(), sizeof(int) * (ncls + 1), cudaMemcpyHostToDevice,
                                  st) ||
                  cudaMemcpyAsync(colo_d, colseg_off.data(), sizeof(int) * (ncls + 1), cudaMemcpyHostToDevice, st) ||
                  cudaMemcpyAsync(cols_d, colseg.data(), sizeof(int) * nseg, cudaMemcpyHostToDevice, st) ||
                  cudaMemcpyAsync(segst_d, seg_start.data(), sizeof(long long) * nseg, cudaMemcpyHostToDevice,
                                  st))))
        return cuda_err("upload");
    P.cls = cls_d;
    P.tab = tab_d;
    P.u = u_d;
    P.v = v_d;
    P.G = G_d;

    cudaEvent_t ev[5];
    for (auto& e : ev) cudaEventCreate(&e);
    struct EvGuard {
        cudaEvent_t* e;
        ~EvGuard()
        {
            for (int i = 0; i < 5; ++i) cudaEventDestroy(e[i]);
        }
    } evg{ev};
    cudaEventRecord(ev[0], st);

    // stage 1: generator rows (scratch: two level buffers, the work buffer, factor samples)
    {
        long long sA = 1, sT = 1, sR = 1;
        for (const A1Class& C : h->cls) {
            for (int l = 0; l <= J; ++l) sA = std::max<long long>(sA, (long long)C.g[0][l].w * C.g[1][l].w);
            for (int l = 0; l < J; ++l) sT = std::max<long long>(sT, 2LL * C.g[0][l].w * C.g[1][l + 1].w);
            sT = std::max<long long>(sT, (long long)(2 * r + 1) * C.g[1][0].w);
            sR = std::max<long long>(sR, C.g[0][0].w + C.g[1][0].w + 4LL * r);
        }
        P.sA = sA;
        P.sT = sT;
        P.sR = sR;
        const long long items = (long long)ncls * m;
        auto kgen = k_a1_generators<D, 0>;
        if (D == 2) {  // 2-D: the common filter lengths with the taps in registers
            if (Lf == 4) kgen = k_a1_generators<D, 4>;
            if (Lf == 6) kgen = k_a1_generators<D, 6>;
            if (Lf == 8) kgen = k_a1_generators<D, 8>;
            if (Lf == 12) kgen = k_a1_generators<D, 12>;
        }
        const ScratchPlan sp = plan_scratch(kgen, items, 2 * sA + sT + sR);
        double* slab = nullptr;
        if (!sp.smem && !db.alloc(&slab, (size_t)sp.grid * (2 * sA + sT + sR))) return oom();
        kgen<<<sp.grid, A1_THREADS, sp.smem ? sp.bytes : 0, st>>>(P, slab);
        count_launch();
        if (cudaMemsetAsync(vmax_d, 0, sizeof(double) * m, st) || cudaMemsetAsync(amax_d, 0, sizeof(double) * m, st))
            return cuda_err("maxima set-up");
        const dim3 gv((unsigned)std::min<int64_t>(256, (N + 255) / 256), m),
            gg((unsigned)std::min<int64_t>(256, (gtotal + 255) / 256), m);
        k_a1_absmax<<<gv, 256, 0, st>>>(v_d, N, N, (unsigned long long*)vmax_d);
        k_a1_absmax<<<gg, 256, 0, st>>>(G_d, gtotal, gtotal, (unsigned long long*)amax_d);
        count_launch(2);
        if (cudaGetLastError() != cudaSuccess) return cuda_err("generator launch");
    }
    cudaEventRecord(ev[1], st);

    // stage 2: thresholds by bisection on the Schur bound (the rule of the oracle's reading)
    std::vector<double> vmax(m), amax(m), eps(m), top(m);
    if (cudaMemcpyAsync(vmax.data(), vmax_d, sizeof(double) * m, cudaMemcpyDeviceToHost, st) ||
        cudaMemcpyAsync(amax.data(), amax_d, sizeof(double) * m, cudaMemcpyDeviceToHost, st) ||
        cudaStreamSynchronize(st))
        return cuda_err("generator stage");
    for (int k = 0; k < m; ++k) {
        eps[k] = vmax[k] > 0.0 ? h->eta / (m * vmax[k]) : 1e300;
        top[k] = amax[k] * (1.0 + 1e-15) + 1e-300;
    }
    double *eps_d = st_d, *top_d = st_d + m, *lo_d = st_d + 2 * m, *hi_d = st_d + 3 * m, *tq_d = st_d + 4 * m,
           *tau_d = st_d + 5 * m;
    if (cudaMemcpyAsync(eps_d, eps.data(), sizeof(double) * m, cudaMemcpyHostToDevice, st) ||
        cudaMemcpyAsync(top_d, top.data(), sizeof(double) * m, cudaMemcpyHostToDevice, st) ||
        cudaMemcpyAsync(tq_d, top.data(), sizeof(double) * m, cudaMemcpyHostToDevice, st) ||
        cudaMemsetAsync(done_d, 0, sizeof(int) * m, st))
        return cuda_err("threshold set-up");
    if (h->rule == PC_ALG1_HARD) {
        // tau_k = eps_k (everything for a zero window)
        if (cudaMemcpyAsync(tau_d, eps.data(), sizeof(double) * m, cudaMemcpyHostToDevice, st))
            return cuda_err("threshold set-up");
    } else {
        const int last = 80;
        int dev = 0, sms = 1;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int grid = (int)std::min<long long>((long long)ncls * m, 8LL * sms);
        for (int step = 0; step <= last; ++step) {
            k_a1_segsum<<<grid, A1_THREADS, 0, st>>>(P, perm_d, segst_d, seglen_d, segrow_d, nseg, tq_d, segsum_d);
            k_a1_bisect<<<m, 256, 0, st>>>(ncls, nseg, segrow_d, colo_d, cols_d, segsum_d, eps_d, top_d, lo_d, hi_d,
                                           tq_d, tau_d, done_d, step, last);
            count_launch(2);
        }
        if (cudaGetLastError() != cudaSuccess) return cuda_err("threshold launch");
    }
    P.tau = tau_d;
    h->tau.assign(m, 0.0);
    std::vector<int> rbox_init(4 * (size_t)ncls);
    for (int c = 0; c < ncls; ++c) {
        rbox_init[4 * c] = rbox_init[4 * c + 2] = INT_MAX;
        rbox_init[4 * c + 1] = rbox_init[4 * c + 3] = INT_MIN;
    }
    if (cudaMemcpyAsync(rbox_d, rbox_init.data(), sizeof(int) * rbox_init.size(), cudaMemcpyHostToDevice, st))
        return cuda_err("support set-up");
    {
        const int grid = (int)std::min<long long>((long long)ncls * m, 1024);
        k_a1_support<D><<<grid, A1_THREADS, 0, st>>>(P, kept_d, rbox_d);
        count_launch();
        if (cudaGetLastError() != cudaSuccess) return cuda_err("support launch");
    }
    std::vector<long long> keptc((size_t)m * ncls);
    std::vector<int> rbox(4 * (size_t)ncls);
    if (cudaMemcpyAsync(h->tau.data(), tau_d, sizeof(double) * m, cudaMemcpyDeviceToHost, st) ||
        cudaMemcpyAsync(keptc.data(), kept_d, sizeof(long long) * keptc.size(), cudaMemcpyDeviceToHost, st) ||
        cudaMemcpyAsync(rbox.data(), rbox_d, sizeof(int) * rbox.size(), cudaMemcpyDeviceToHost, st) ||
        cudaStreamSynchronize(st))
        return cuda_err("threshold stage");
    cudaEventRecord(ev[2], st);

    // product boxes: R per class (the union of the kept supports, or the period), its chain
    h->kept.assign(m, 0);
    int64_t ftotal = 0, ttotal = 0;
    long long sA = 1, sT = 1;
    for (int c = 0; c < ncls; ++c) {
        A1Class& C = h->cls[c];
        long long any = 0;
        for (int k = 0; k < m; ++k) {
            any += keptc[(size_t)k * ncls + c];
            h->kept[k] += keptc[(size_t)k * ncls + c] * h->rows;
        }
        if (!any) {
            C.rsize = C.tlen = 0;
            C.foff = ftotal;
            C.toff = ttotal;
            continue;
        }
        Ax b0[2];
        for (int d = 0; d < 2; ++d) {
            if (d >= D) {
                b0[d] = {0, 1};
                continue;
            }
            const long long lo = rbox[4 * c + 2 * d], hi = rbox[4 * c + 2 * d + 1];
            b0[d] = (hi - lo + 1 >= n) ? Ax{0, n} : Ax{(int)lo, (int)(hi - lo + 1)};
        }
        C.tlen = chain(D, n, J, Lf, b0, C.c, C.coffl);
        C.rsize = b0[0].w * b0[1].w;
        C.foff = ftotal;
        C.toff = ttotal;
        ftotal += (int64_t)m * C.rsize;
        ttotal += (int64_t)h->rows * C.tlen;
        for (int l = 0; l <= J; ++l) sA = std::max<long long>(sA, (long long)C.c[0][l].w * C.c[1][l].w);
        for (int l = 0; l < J; ++l) sT = std::max<long long>(sT, 2LL * C.c[0][l].w * C.c[1][l + 1].w);
    }
    h->nnz = ttotal;
    const size_t esz = h->fp32 ? sizeof(float) : sizeof(double);
    if (h->fp32) {
        if (!db.alloc(&P.Fb32, ftotal)) return oom();
    } else if (!db.alloc(&P.Fb, ftotal)) {
        return oom();
    }
    {
        // per-pixel lists of the nonzero windows (a hat window is nonzero on a few of the m)
        int* cnt_d;
        int slots = 0;
        if (!db.alloc(&cnt_d, 1)) return oom();
        if (cudaMemsetAsync(cnt_d, 0, sizeof(int), st)) return cuda_err("window lists");
        k_a1_wlist<<<1024, 256, 0, st>>>(v_d, m, N, 0, cnt_d, nullptr, nullptr, nullptr);
        if (cudaMemcpyAsync(&slots, cnt_d, sizeof(int), cudaMemcpyDeviceToHost, st) || cudaStreamSynchronize(st))
            return cuda_err("window lists");
        slots = std::max(slots, 1);
        int* wk;
        double* wv64 = nullptr;
        float* wv32 = nullptr;
        if (!db.alloc(&wk, (size_t)slots * N) ||
            (h->fp32 ? !db.alloc(&wv32, (size_t)slots * N) : !db.alloc(&wv64, (size_t)slots * N)))
            return oom();
        k_a1_wlist<<<1024, 256, 0, st>>>(v_d, m, N, slots, cnt_d, wk, wv64, wv32);
        count_launch(2);
        P.wslots = slots;
        P.wk = wk;
        P.wv64 = wv64;
        P.wv32 = wv32;
    }
    // Theta~ storage; with PC_ALG1_DISCARD one buffer of at most 8 GB (or the largest class) that
    // every group of classes overwrites in turn
    int64_t tcap = std::max<int64_t>(ttotal, 1);
    if (h->discard) {
        int64_t big = 1;
        for (const A1Class& C : h->cls) big = std::max<int64_t>(big, (int64_t)h->rows * C.tlen);
        tcap = std::max(big, std::min<int64_t>(tcap, (int64_t)(8LL << 30) / (int64_t)esz));
    }
    if (cudaMalloc(&h->theta_d, esz * tcap) != cudaSuccess) {
        h->theta_d = nullptr;
        (void)cudaGetLastError();
        return oom();
    }
    if (cudaMemcpyAsync(cls_d, h->cls.data(), sizeof(A1Class) * ncls, cudaMemcpyHostToDevice, st))
        return cuda_err("class upload");
    if (h->fp32)
        P.theta32 = (float*)h->theta_d;
    else
        P.theta = (double*)h->theta_d;
    P.sA = sA;
    P.sT = sT;
    P.sR = 0;

    // stage 3: F~ per (class, term); stage 4: the rows of Theta~
    {
        const ScratchPlan sp = plan_scratch(k_a1_synth<D>, (long long)ncls * m, 2 * sA + sT);
        double* slab = nullptr;
        if (!sp.smem && !db.alloc(&slab, (size_t)sp.grid * (2 * sA + sT))) return oom();
        k_a1_synth<D><<<sp.grid, A1_THREADS, sp.smem ? sp.bytes : 0, st>>>(P, slab);
        count_launch();
        if (cudaGetLastError() != cudaSuccess) return cuda_err("synthesis launch");
    }
    cudaEventRecord(ev[3], st);
    {
        // up to three launches: the classes whose buffers fit in 100 KB of shared memory (two
        // CTAs per SM), in 200 KB (one), and the others with a global slab per CTA
        const size_t esz4 = h->fp32 ? sizeof(float) : sizeof(double);
        std::vector<int> lists[3];
        long long mA[3] = {1, 1, 1}, mT[3] = {1, 1, 1};
        for (int c = 0; c < ncls; ++c) {
            const A1Class& C = h->cls[c];
            if (!C.tlen) continue;
            long long cA = 1, cT = 1;
            for (int l = 0; l <= J; ++l) cA = std::max<long long>(cA, (long long)C.c[0][l].w * C.c[1][l].w);
            for (int l = 0; l < J; ++l) cT = std::max<long long>(cT, 2LL * C.c[0][l].w * C.c[1][l + 1].w);
            const size_t need = (size_t)(2 * cA + cT) * esz4;
            const int w = need <= 100 * 1024 ? 0 : need <= 200 * 1024 ? 1 : 2;
            lists[w].push_back(c);
            mA[w] = std::max(mA[w], cA);
            mT[w] = std::max(mT[w], cT);
        }
        auto kern32 = k_a1_product<D, float, 0>;
        if (D == 2) {
            // FP32 2-D products for the common filter lengths with the taps in registers
            if (Lf == 4) kern32 = k_a1_product<D, float, 4>;
            if (Lf == 6) kern32 = k_a1_product<D, float, 6>;
            if (Lf == 8) kern32 = k_a1_product<D, float, 8>;
            if (Lf == 12) kern32 = k_a1_product<D, float, 12>;
        }
        // groups of consecutive classes whose rows fit the Theta~ buffer (one group unless discarding)
        std::vector<int> group(ncls, 0);
        std::vector<int64_t> gbase(1, 0);
        {
            int64_t used = 0;
            for (int c = 0; c < ncls; ++c) {
                const int64_t sz = (int64_t)h->rows * h->cls[c].tlen;
                if (used + sz > tcap && used > 0) {
                    gbase.push_back(h->cls[c].toff);
                    used = 0;
                }
                group[c] = (int)gbase.size() - 1;
                used += sz;
            }
        }
        std::vector<int> order;
        std::vector<std::array<int64_t, 3>> runs;  // (group, tier, start in order)
        for (int g = 0; g < (int)gbase.size(); ++g)
            for (int w = 0; w < 3; ++w) {
                const size_t start = order.size();
                for (int c : lists[w])
                    if (group[c] == g) order.push_back(c);
                if (order.size() > start) runs.push_back({g, w, (int64_t)start});
            }
        int* order_d = nullptr;
        if (!db.alloc(&order_d, order.size())) return oom();
        if (!order.empty() &&
            cudaMemcpyAsync(order_d, order.data(), sizeof(int) * order.size(), cudaMemcpyHostToDevice, st))
            return cuda_err("class list");
        for (size_t ri = 0; ri < runs.size(); ++ri) {
            const int g = (int)runs[ri][0], w = (int)runs[ri][1];
            const int64_t start = runs[ri][2];
            const int64_t end = ri + 1 < runs.size() ? runs[ri + 1][2] : (int64_t)order.size();
            int* cl_d = order_d + start;
            P.tbase = gbase[g];
            P.sA = mA[w];
            P.sT = mT[w];
            const long long per = 2 * mA[w] + mT[w];
            const int nl = (int)(end - start);
            const long long items = (long long)nl * h->rows;
            if (h->fp32) {
                const ScratchPlan sp = plan_scratch(kern32, items, per, sizeof(float));
                float* slab = nullptr;
                if (!sp.smem && !db.alloc(&slab, (size_t)sp.grid * per)) return oom();
                kern32<<<sp.grid, A1_THREADS, sp.smem ? sp.bytes : 0, st>>>(P, cl_d, nl, slab);
            } else {
                const ScratchPlan sp = plan_scratch(k_a1_product<D, double>, items, per);
                double* slab = nullptr;
                if (!sp.smem && !db.alloc(&slab, (size_t)sp.grid * per)) return oom();
                k_a1_product<D, double><<<sp.grid, A1_THREADS, sp.smem ? sp.bytes : 0, st>>>(P, cl_d, nl, slab);
            }
            count_launch();
        }
        if (cudaGetLastError() != cudaSuccess) return cuda_err("product launch");
    }
    cudaEventRecord(ev[4], st);
    if (cudaStreamSynchronize(st) != cudaSuccess) return cuda_err("Algorithm 1");
    for (int i = 0; i < 4; ++i) {
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, ev[i], ev[i + 1]);
        h->stage_ms[i] = ms;
    }
    return PC_OK;
}

}  // namespace

extern "C" {

pc_status pc_alg1_create(const pc_desc* desc, const double* u, const double* v, double eta, int rule, int flags,
                         void* stream, pc_alg1_handle* out)
{
    if (!desc || !u || !v || !out || !(eta >= 0.0) || !std::isfinite(eta) ||
        (rule != PC_ALG1_SCHUR && rule != PC_ALG1_HARD) || (flags & ~PC_ALG1_DISCARD))
        return fail(nullptr, PC_ERR_INVALID_ARG,
                    "pc_alg1_create: NULL pointer, eta not finite and >= 0, an unknown rule or flag");
    *out = nullptr;
    const pc_desc& d = *desc;
    if ((d.dim != 1 && d.dim != 2) || d.n < 2 || (d.n & (d.n - 1)) || d.levels < 1 ||
        d.levels > pcw::alg1::A1_MAXJ || (d.n >> d.levels) < 1 || d.delta < 1 || d.delta > 10 || d.m < 1 ||
        d.m > 256 || d.radius < 0 || 2 * d.radius + 1 > d.n || (d.family != 0 && d.family != 1))
        return fail(nullptr, PC_ERR_INVALID_ARG, "pc_alg1_create: descriptor out of range");
    if (d.order != PC_ORDER_MULT_THEN_CONV)
        return fail(nullptr, PC_ERR_UNSUPPORTED,
                    "pc_alg1_create: only the paper's order (the other is the transpose with flipped kernels)");
    if (d.precision != PC_FP64 && d.precision != PC_FP32)
        return fail(nullptr, PC_ERR_INVALID_ARG, "pc_alg1_create: unknown precision");
    if (d.dim * d.levels > 16) return fail(nullptr, PC_ERR_UNSUPPORTED, "pc_alg1_create: more than 2^16 classes");
    pc_alg1* h = new (std::nothrow) pc_alg1;
    if (!h) return fail(nullptr, PC_ERR_OOM, "pc_alg1_create: host allocation failed");
    h->D = d.dim;
    h->n = d.n;
    h->J = d.levels;
    h->Lf = 2 * d.delta;
    h->m = d.m;
    h->r = d.radius;
    h->nJ = d.n >> d.levels;
    h->rows = (d.dim == 2) ? h->nJ * h->nJ : h->nJ;
    h->ncls = 1 << (d.dim * d.levels);
    h->N = (d.dim == 2) ? (int64_t)d.n * d.n : d.n;
    h->eta = eta;
    h->fp32 = d.precision == PC_FP32;
    h->rule = rule;
    h->discard = (flags & PC_ALG1_DISCARD) != 0;
    pc_status s = (d.dim == 2) ? alg1_run<2>(h, desc, u, v, (cudaStream_t)stream)
                               : alg1_run<1>(h, desc, u, v, (cudaStream_t)stream);
    if (s != PC_OK) {
        pc_alg1_destroy(h);
        return s;
    }
    *out = h;
    return PC_OK;
}

pc_status pc_alg1_info(pc_alg1_handle h, int64_t* nnz, double* tau, int64_t* kept, double* stage_ms)
{
    if (!h) return fail(nullptr, PC_ERR_INVALID_ARG, "pc_alg1_info: NULL handle");
    if (nnz) *nnz = h->nnz;
    for (int k = 0; k < h->m; ++k) {
        if (tau) tau[k] = h->tau[k];
        if (kept) kept[k] = h->kept[k];
    }
    if (stage_ms)
        for (int i = 0; i < 4; ++i) stage_ms[i] = h->stage_ms[i];
    return PC_OK;
}

// Class, translate and the columns of row mu (canonical) of Theta~; vals from the row's stored
// values `row` (host).  Returns the entry count.
static int64_t alg1_row_entries(const pc_alg1* h, int64_t mu, const std::vector<BandId>& bands, int* cls_out,
                                int64_t* toff_out, const double* row, int64_t* cols, double* vals)
{
    const int D = h->D, n = h->n, J = h->J, nJ = h->nJ;
    size_t b = 0;
    while (b + 1 < bands.size() && bands[b + 1].off <= mu) ++b;
    const int j = bands[b].j, nl = n >> j, ph = 1 << (J - j);
    const int64_t pos = mu - bands[b].off;
    const int x0 = (D == 2) ? (int)(pos / nl) : (int)pos, x1 = (D == 2) ? (int)(pos % nl) : 0;
    const int c = h->band_cbase[b] + (D == 2 ? (x0 & (ph - 1)) * ph + (x1 & (ph - 1)) : (x0 & (ph - 1)));
    const int t0 = x0 >> (J - j), t1 = (D == 2) ? x1 >> (J - j) : 0;
    const A1Class& C = h->cls[c];
    if (cls_out) *cls_out = c;
    if (toff_out) *toff_out = C.toff + (int64_t)(D == 2 ? t0 * nJ + t1 : t0) * C.tlen;
    if (!cols) return C.tlen;
    int64_t k = 0;
    if (C.tlen)
        host_segments(D, J, C.c, C.coffl, [&](int band, int l, int, int, int off, Ax b0, Ax b1) {
            const int nlb = n >> l, sh = J - l;
            for (int i0 = 0; i0 < b0.w; ++i0)
                for (int i1 = 0; i1 < b1.w; ++i1) {
                    const int y0 = (b0.a + i0 + (t0 << sh)) & (nlb - 1);
                    const int y1 = (D == 2) ? ((b1.a + i1 + (t1 << sh)) & (nlb - 1)) : 0;
                    cols[k] = bands[band].off + (D == 2 ? (int64_t)y0 * nlb + y1 : y0);
                    if (vals) vals[k] = row[off + i0 * b1.w + i1];
                    ++k;
                }
        });
    return k;
}

// Copies n values of Theta~ from element offset `off` of the device array into host doubles.
static cudaError_t alg1_copy_values(const pc_alg1* h, int64_t off, int64_t n, double* out)
{
    if (n <= 0) return cudaSuccess;
    if (h->fp32) {
        std::vector<float> tf((size_t)n);
        const cudaError_t e = cudaMemcpy(tf.data(), (const float*)h->theta_d + off, sizeof(float) * n,
                                         cudaMemcpyDeviceToHost);
        for (int64_t i = 0; i < n; ++i) out[i] = tf[(size_t)i];
        return e;
    }
    return cudaMemcpy(out, (const double*)h->theta_d + off, sizeof(double) * n, cudaMemcpyDeviceToHost);
}

pc_status pc_alg1_export(pc_alg1_handle h, int64_t* row_ptr, int64_t* cols, double* vals)
{
    if (!h || !row_ptr || (h->nnz && (!cols || !vals)))
        return fail(nullptr, PC_ERR_INVALID_ARG, "pc_alg1_export: NULL pointer");
    if (h->discard) return fail(nullptr, PC_ERR_UNSUPPORTED, "pc_alg1_export: Theta~ was not kept");
    std::vector<double> t((size_t)h->nnz);
    if (alg1_copy_values(h, 0, h->nnz, t.data()) != cudaSuccess)
        return fail(nullptr, PC_ERR_CUDA, "pc_alg1_export: copy failed");
    const std::vector<BandId> bands = canonical_bands(h->D, h->n, h->J);
    int64_t pos = 0;
    row_ptr[0] = 0;
    for (int64_t mu = 0; mu < h->N; ++mu) {
        int64_t toff = 0;
        alg1_row_entries(h, mu, bands, nullptr, &toff, nullptr, nullptr, nullptr);
        pos += alg1_row_entries(h, mu, bands, nullptr, nullptr, t.data() + toff, cols + pos, vals + pos);
        row_ptr[mu + 1] = pos;
    }
    return PC_OK;
}

pc_status pc_alg1_row(pc_alg1_handle h, int64_t row, int64_t* cols, double* vals, int64_t* count)
{
    if (!h || !count || row < 0 || row >= h->N)
        return fail(nullptr, PC_ERR_INVALID_ARG, "pc_alg1_row: NULL handle or count, or row out of range");
    if (h->discard) return fail(nullptr, PC_ERR_UNSUPPORTED, "pc_alg1_row: Theta~ was not kept");
    const std::vector<BandId> bands = canonical_bands(h->D, h->n, h->J);
    int64_t toff = 0;
    const int64_t len = alg1_row_entries(h, row, bands, nullptr, &toff, nullptr, nullptr, nullptr);
    if (!cols && !vals) {
        *count = len;
        return PC_OK;
    }
    if (!cols || !vals || *count < len)
        return fail(nullptr, PC_ERR_INVALID_ARG, "pc_alg1_row: buffers missing or shorter than the row");
    std::vector<double> t((size_t)len);
    if (alg1_copy_values(h, toff, len, t.data()) != cudaSuccess)
        return fail(nullptr, PC_ERR_CUDA, "pc_alg1_row: copy failed");
    *count = alg1_row_entries(h, row, bands, nullptr, nullptr, t.data(), cols, vals);
    return PC_OK;
}

void pc_alg1_destroy(pc_alg1_handle h)
{
    if (!h) return;
    if (h->theta_d) cudaFree(h->theta_d);
    delete h;
}

}  // extern "C"
