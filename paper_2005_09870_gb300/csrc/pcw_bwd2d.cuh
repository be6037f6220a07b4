// 2-D backward: adjoint of the row assembly, in three phases.
//
//   phase 1 (k_backward_queue, persistent; k_backward2d per band for FP64): per stored row s,
//           dL/ds on the row's region by the transposed localized transform of the row's
//           dL/dTheta entries, written to the scratch S (band b at Soff[b], row rl at
//           + rl * RR_b, region row-major);
//   phase 2 (k_bwd_dv4, k_bwd_dv for FP64): dL/dv_k(x) = sum_b sum_{rows l covering x}
//           F_{k,b}(x - t_l) S_{b,l}(x - t_l), a gather (no atomics), one thread per pixel;
//   phase 3 (k_bwd_dF_wl, k_bwd_dF without window lists): dL/dF_{k,b}(q) =
//           sum_l v_k(t_l + q) S_{b,l}(q), chunks of rows per CTA, one atomic per (k, q, chunk).
// The adjoint of F = kappa_k * rho_b (dL/dkappa_k) then runs in k_dfilt_pass2 / pass1.
#pragma once
#include "pcw_asm2d.cuh"

namespace pcw {

// Transpose of pass_hg along one axis: for every input position p (unwrapped ri.lo + p),
//   in_bar[p] = sum_i h[i] yl_bar(C) [2C + i = X]  +  sum_i g[i] yh_bar(C) [2C + 2 - LF + i = X]
// with C - ro.lo in [0, ro.cnt) (or modulo the output length when the output is full).
// Work items are chunks of 2*CH inputs starting at an even unwrapped position.
// exact (the filter fills the template, Lf == LF): the outputs ro of a non-wrapping input
// range ri are exactly the C that the kept positions read, so the window loads need no bounds
// checks; the positions of a line's last chunk past ri read up to ADJ_SLACK elements (lines)
// beyond its end, which must lie inside the arena, and are discarded.
constexpr int ADJ_SLACK = 2 * PASS_CH;
template <typename T, int LF, int CH>
__device__ __forceinline__ void pass_hg_adj(const T* yl, const T* yh, int olstride, int ostride, Range ro, int n_out,
                                            T* out, int lstride, int stride, Range ri, int nlines,
                                            const T (&hr)[LF], const T (&gr)[LF], int tid, int gt, bool exact)
{
    constexpr int WL = CH + LF / 2 - 1;
    const int xs = ri.lo & ~1;               // first chunk start (even, unwrapped)
    const int nch = (ri.lo + ri.cnt - xs + 2 * CH - 1) / (2 * CH);
    const int items = nlines * nch;
    Stepper st;
    st.init(tid, gt, nlines);
    const int nom = n_out - 1;
    for (int it = tid; it < items; it += gt, st.next()) {
        const int line = st.b;
        const int X0 = xs + st.a * 2 * CH;
        const int h0 = (X0 >> 1) - LF / 2 + 1 - ro.lo;  // window of yl_bar starts at C = X0/2 - LF/2 + 1
        const int g0 = (X0 >> 1) - ro.lo;               // window of yh_bar starts at C = X0/2
        const T* ylr = yl + line * olstride;
        const T* yhr = yh + line * olstride;
        T wl[WL], wh[WL];
        if (exact && !ro.full) {
            const T* pl = ylr + h0 * ostride;
            const T* ph = yhr + g0 * ostride;
#pragma unroll
            for (int t = 0; t < WL; ++t) {
                wl[t] = pl[t * ostride];
                wh[t] = ph[t * ostride];
            }
        } else {
#pragma unroll
            for (int t = 0; t < WL; ++t) {
                int cl = h0 + t, ch = g0 + t;
                if (ro.full) {
                    cl &= nom;
                    ch &= nom;
                    wl[t] = ylr[cl * ostride];
                    wh[t] = yhr[ch * ostride];
                } else {
                    wl[t] = ((unsigned)cl < (unsigned)ro.cnt) ? ylr[cl * ostride] : T(0);
                    wh[t] = ((unsigned)ch < (unsigned)ro.cnt) ? yhr[ch * ostride] : T(0);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < CH; ++u) {
#pragma unroll
            for (int par = 0; par < 2; ++par) {
                T acc = T(0);
#pragma unroll
                for (int m = 0; m < LF / 2; ++m) {
                    acc = fma(hr[2 * m + par], wl[u - m + LF / 2 - 1], acc);
                    acc = fma(gr[2 * m + par], wh[u + LF / 2 - 1 - m], acc);
                }
                const int p = X0 + 2 * u + par - ri.lo;
                if ((unsigned)p < (unsigned)ri.cnt) out[line * lstride + p * stride] = acc;
            }
        }
    }
}

// Transpose of pass_lo (scaling filter f of length len at stride S, offsets [0, len)).
template <typename T>
__device__ __forceinline__ void pass_lo_adj(const T* y, int olstride, int ostride, Range ro, int n_out, T* out,
                                            int lstride, int stride, Range ri, int nlines, const T* f, int len, int S,
                                            int tid, int gt)
{
    const int items = nlines * ri.cnt;
    Stepper st;
    st.init(tid, gt, nlines);
    const int nom = n_out - 1;
    for (int it = tid; it < items; it += gt, st.next()) {
        const int line = st.b, p = st.a;
        const int X = ri.lo + p;
        const T* yr = y + line * olstride;
        T acc = T(0);
        for (int i = X & (S - 1); i < len; i += S) {
            int c = ((X - i) >> log2i(S)) - ro.lo;
            if (ro.full)
                c &= nom;
            else if ((unsigned)c >= (unsigned)ro.cnt)
                continue;
            acc = fma(f[i], yr[c * ostride], acc);
        }
        out[line * lstride + p * stride] = acc;
    }
}

// Scatters the stencil window of one column band from the row's dL/dTheta into a zeroed
// coefficient array (transpose of write_win).
template <typename T>
__device__ __forceinline__ void read_win(const OpDev<T>& op, const T* __restrict__ Gr, T* Zb, int pz, Range r0,
                                         Range r1, int nj, int f0, int W0, int f1, int W1, int64_t src, int tid,
                                         int gt)
{
    const int tot = W0 * W1;
    if (tot <= 0) return;
    const T* g = Gr + src;
    if (!r0.full && !r1.full && op.gap >= 0) {
        T* z = Zb + (f0 - r0.lo) * pz + (f1 - r1.lo);
        // asynchronous copies (cp.async): every copy of the thread in flight at once, no register
        // round trip; read_level waits for them.  Positions stepped without divisions.
        WinStep ws;
        ws.init(tid, gt, pz, W1);
        for (int i = tid; i < tot; i += gt) {
            const unsigned dst = (unsigned)__cvta_generic_to_shared(z + ws.zi);
            if constexpr (sizeof(T) == 4)
                asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(g + i) : "memory");
            else
                asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(g + i) : "memory");
            ws.next();
        }
    } else {
        Stepper st;
        st.init(tid, gt, W1);
        for (int idx = tid; idx < tot; idx += gt, st.next()) {
            const int p0 = pmod(f0 + st.a - r0.lo, nj), p1 = pmod(f1 + st.b - r1.lo, nj);
            if ((r0.full || p0 < r0.cnt) && (r1.full || p1 < r1.cnt)) Zb[p0 * pz + p1] = g[idx];
        }
    }
}

// Fills Z = [LL | (0,1) | (1,0) | (1,1)] of level jj from the row's dL/dTheta: detail bands
// always, LL (the approximation band) when jj == L; other LL entries are left as they are.
template <typename T>
__device__ __forceinline__ void read_level(const OpDev<T>& op, const Row2& R, const int* meta, const T* Gth, T* Z,
                                           Range q0r, Range q1r, int jj, int tid, int gt)
{
    const int n = op.n, L = op.L, dense = op.gap < 0;
    const int zq = q0r.cnt * q1r.cnt, nj = n >> jj;
    const int tmax = (jj == L) ? 4 : 3;
    for (int t = 0; t < tmax; ++t) {
        const int b2 = (t == 3) ? 0 : band_of_level(2, L, jj, t);
        const int e0 = (t == 3) ? 0 : (t >= 1 ? 1 : 0), e1 = (t == 3) ? 0 : (t == 1 ? 0 : 1);
        (void)e0;
        (void)e1;
        (void)dense;
        const int* w = meta + WIN_OFF + 4 * b2;
        const int f0 = w[0], W0 = w[1], f1 = w[2], W1 = w[3];
        read_win(op, Gth, Z + ((t == 3) ? 0 : (1 + t) * zq), q1r.cnt, q0r, q1r, nj, f0, W0, f1, W1,
                 R.row_base + meta[b2], tid, gt);
    }
    asm volatile("cp.async.wait_all;" ::: "memory");  // this thread's window copies have landed
}

// Phase 1, one stored 2-D row by one thread group (same plan, arenas and filter area as the
// forward).  Writes dL/ds of the row to Sout + Sband + rl * RR and its active-term mask.
template <typename T, int LF>
__device__ __forceinline__ void bwd2d_row(const OpDev<T>& op, const AsmCfg& cfg, int rl, const T* fS, int* meta,
                                          T* arena, int gid, int tid, const T* __restrict__ Gth,
                                          T* __restrict__ Sout, int64_t Sband,
                                          unsigned long long* __restrict__ amask_out)
{
    constexpr int CH = 4;
    const int gt = cfg.gt;
    const int n = op.n, Lf = op.Lf;
    T* const arena_end = arena + cfg.arena;
    const int A = cfg.arena;
    const int k0_band = (op.gap < 0) ? 0 : max(1, band_info(2, n, op.L, cfg.b).j - op.gap) - 1;
    const int lenk = (k0_band > 0) ? wav_len(k0_band, Lf) : 0;
    const Row2 R = row2_setup(op, cfg.b, rl);
    if (!row2_meta(op, R, cfg.b, meta, tid, gt, gid, amask_out != nullptr)) return;
    const int k0 = R.k0;
    (void)k0_band;

    T hr[LF], gr[LF];
#pragma unroll
    for (int i = 0; i < LF; ++i) {
        hr[i] = fS[i];
        gr[i] = fS[LF + i];
    }
    const T* phiS = fS + 2 * LF;
    const Range A0 = R.A0, A1 = R.A1;
    const int RR = A0.cnt * A1.cnt;
    const int B = max(1, min(cfg.batch, A0.cnt));
    const int lv0 = (k0 == 0) ? 1 : k0;
    if (amask_out && tid < op.mwords) {  // active terms of this row as a bit mask (for phase 3)
        const unsigned char* act = reinterpret_cast<const unsigned char*>(meta + ACT_OFF);
        unsigned long long w = 0ull;
        for (int t = 0; t < meta[NACT_OFF]; ++t)
            if ((act[t] >> 6) == tid) w |= 1ull << (act[t] & 63);
        amask_out[R.srow * op.mwords + tid] = w;
    }

    // forward ranges per level (inputs p*, outputs q*): recomputed from the region
    Range P0[MAXL + 2], P1[MAXL + 2];  // P*[jj] = output range of level jj
    {
        Range p0 = A0, p1 = A1;
        for (int jj = lv0; jj <= R.jhi; ++jj) {
            const bool lo_only = (jj == lv0) && k0 > 0;
            const int nj = n >> jj, S = lo_only ? (1 << k0) : 2;
            P0[jj] = lo_only ? range_filter(A0, S, 0, lenk, nj) : range_cascade(p0, Lf, nj);
            P1[jj] = pad_odd(lo_only ? range_filter(A1, S, 0, lenk, nj) : range_cascade(p1, Lf, nj), nj);
            p0 = P0[jj];
            p1 = P1[jj];
        }
    }
    // coarse to fine: Z (level jj) -> Y -> X (LL of level jj-1, which is Z's LL next)
    for (int jj = R.jhi; jj >= lv0; --jj) {
        const bool first = (jj == lv0);
        const bool lo_only = first && k0 > 0;
        const int nj = n >> jj;
        const int S = lo_only ? (1 << k0) : 2;
        const Range q0r = P0[jj], q1r = P1[jj];
        const Range p0 = first ? A0 : P0[jj - 1], p1 = first ? A1 : P1[jj - 1];
        const int n_in = first ? n : (n >> (jj - 1));
        const int zq = q0r.cnt * q1r.cnt;
        const int zsz = (lo_only ? 1 : 4) * zq;
        const int ysz = (lo_only ? 1 : 2) * p0.cnt * q1r.cnt;
        const int xsz = first ? B * A1.cnt : p0.cnt * p1.cnt;
        // Y sits ADJ_SLACK below the arena end; the column reads of Z run up to ADJ_SLACK rows
        // past it (see pass_hg_adj)
        if (zsz + ysz + ADJ_SLACK > A || xsz + ysz + ADJ_SLACK > A || zsz + ADJ_SLACK * q1r.cnt > A) {
            flag_error(op.err, ERR_ARENA);
            return;
        }
        if (!lo_only) {
            // LL: zero at the top level (it only feeds coarser levels, which are not kept)
            const int zstart = (jj == R.jhi) ? 0 : zq;
            for (int e = tid; e < 4 * zq - zstart; e += gt) arena[zstart + e] = T(0);
            group_sync(gt, gid);
            read_level(op, R, meta, Gth, arena, q0r, q1r, jj, tid, gt);
            group_sync(gt, gid);
        }
        T* Yl = arena_end - ADJ_SLACK - ysz;
        T* Yh = Yl + p0.cnt * q1r.cnt;
        const bool exact = (Lf == LF);
        // transpose of axis 0 (lines: columns of Y)
        if (lo_only)
            pass_lo_adj<T>(arena, 1, q1r.cnt, q0r, nj, Yl, 1, q1r.cnt, A0, q1r.cnt, phiS, lenk, S, tid, gt);
        else {
#pragma unroll 1
            for (int h2 = 0; h2 < 2; ++h2)
                pass_hg_adj<T, LF, CH>(arena + (h2 ? zq : 0), arena + (h2 ? 3 * zq : 2 * zq), 1, q1r.cnt, q0r, nj,
                                       h2 ? Yh : Yl, 1, q1r.cnt, p0, q1r.cnt, hr, gr, tid, gt, exact);
        }
        group_sync(gt, gid);
        // transpose of axis 1 (lines: rows of Y)
        if (!first) {
            pass_hg_adj<T, LF, CH>(Yl, Yh, q1r.cnt, 1, q1r, nj, arena, p1.cnt, 1, p1, p0.cnt, hr, gr, tid, gt, exact);
            group_sync(gt, gid);
        } else {
            // dL/ds rows in batches, then copied to the scratch
            T* Srow = Sout + Sband + (int64_t)rl * RR;
            for (int r0 = 0; r0 < A0.cnt; r0 += B) {
                const int nr = min(B, A0.cnt - r0);
                if (lo_only)
                    pass_lo_adj<T>(Yl + r0 * q1r.cnt, q1r.cnt, 1, q1r, nj, arena, A1.cnt, 1, A1, nr, phiS, lenk, S,
                                   tid, gt);
                else
                    pass_hg_adj<T, LF, CH>(Yl + r0 * q1r.cnt, Yh + r0 * q1r.cnt, q1r.cnt, 1, q1r, nj, arena, A1.cnt,
                                           1, A1, nr, hr, gr, tid, gt, exact);
                group_sync(gt, gid);
                for (int e = tid; e < nr * A1.cnt; e += gt) Srow[r0 * A1.cnt + e] = arena[e];
                group_sync(gt, gid);
            }
            (void)n_in;
        }
    }
}

// Phase 1 as one launch per row band.
template <typename T, int LF>
__global__ void __launch_bounds__(256, 2) k_backward2d(const __grid_constant__ OpDev<T> op, const AsmCfg cfg,
                                                       const T* __restrict__ Gth, T* __restrict__ Sout,
                                                       const int64_t Sband, unsigned long long* __restrict__ amask_out)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int gt = cfg.gt;
    const int gid = threadIdx.x / gt, tid = threadIdx.x - gid * gt;
    T* fS = reinterpret_cast<T*>(smem_raw);
    int* meta = reinterpret_cast<int*>(smem_raw + sizeof(T) * cfg.filt) + gid * META_INTS;
    T* arena = reinterpret_cast<T*>(smem_raw + sizeof(T) * cfg.filt + sizeof(int) * cfg.rpc * META_INTS) +
               (int64_t)gid * cfg.arena;
    load_filters2d<T, LF>(op, cfg.b, fS);
    __syncthreads();
    const int rloc = blockIdx.x * cfg.rpc + gid;
    if (rloc >= cfg.rows) return;
    bwd2d_row<T, LF>(op, cfg, cfg.row0 + rloc, fS, meta, arena, gid, tid, Gth, Sout, Sband, amask_out);
}

// Phase 1 through the persistent work queue of the forward (FP32): one launch over all bands.
struct BwdQueue {
    const float* G;
    float* S;
    unsigned long long* amask;
    int64_t Soff[MAXB];
};

template <int LF>
__global__ void __launch_bounds__(256, 2) k_backward_queue(const OpDev<float>* __restrict__ opd,
                                                           const BatchItem* __restrict__ items, int nitems,
                                                           int* __restrict__ counter, const __grid_constant__ BwdQueue bq)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ OpDev<float> op_s;
    __shared__ BatchItem it_s;
    __shared__ int idx_s;
    {
        const int* src = reinterpret_cast<const int*>(opd);
        int* dst = reinterpret_cast<int*>(&op_s);
        for (int i = threadIdx.x; i < (int)(sizeof(OpDev<float>) / sizeof(int)); i += blockDim.x) dst[i] = src[i];
    }
    for (;;) {
        if (threadIdx.x == 0) idx_s = atomicAdd(counter, 1);
        __syncthreads();
        const int idx = idx_s;
        if (idx >= nitems) return;
        if (threadIdx.x == 0) it_s = items[idx];
        __syncthreads();
        const AsmCfg cfg = it_s.cfg;
        float* fS = reinterpret_cast<float*>(smem_raw);
        load_filters2d<float, LF>(op_s, cfg.b, fS);
        __syncthreads();
        const int gt = cfg.gt;
        const int gid = threadIdx.x / gt, tid = threadIdx.x - gid * gt;
        if (gid < cfg.rpc) {
            int* meta = reinterpret_cast<int*>(smem_raw + sizeof(float) * cfg.filt) + gid * META_INTS;
            float* arena = reinterpret_cast<float*>(smem_raw + sizeof(float) * cfg.filt +
                                                    sizeof(int) * cfg.rpc * META_INTS) +
                           (int64_t)gid * cfg.arena;
            const int64_t Sband = bq.Soff[cfg.b];
            for (int rb = 0; rb < cfg.rows; rb += cfg.rpc) {
                const int rloc = rb + gid;
                if (rloc >= cfg.rows) break;
                const int rl = cfg.row0 + rloc;
                bwd2d_row<float, LF>(op_s, cfg, rl, fS, meta, arena, gid, tid, bq.G, bq.S, Sband, bq.amask);
                group_sync(gt, gid);
            }
        }
        __syncthreads();
    }
}

// Per-band geometry for phases 2 and 3.
struct BwdBand {
    int j, nj, P0, P1, R0, R1;  // region start offsets (off - r) and folded sizes
    int64_t Soff, Foff, rowoff;  // rowoff: canonical index of the band's first row
    int64_t FToff;               // band offset in the term-contiguous copy of F
};
struct BwdDev {
    int n, m, nb, mp;  // mp: m rounded up to a multiple of 4 (stride of the copy of F)
    int64_t N;
    BwdBand band[MAXB];
};

// Copy of F grouped by 4 terms for the gathers: FT[band][k/4][q][k%4] (terms padded to mp with
// zeros), so that consecutive region positions read consecutive float4s.
__global__ void k_transpose_F(const __grid_constant__ BwdDev bd, const float* __restrict__ F, float* __restrict__ FT)
{
    const int b = blockIdx.y;
    const BwdBand& B = bd.band[b];
    const int RR = B.R0 * B.R1;
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= RR) return;
    for (int k = 0; k < bd.mp; ++k)
        FT[B.FToff + ((int64_t)(k >> 2) * RR + q) * 4 + (k & 3)] = (k < bd.m) ? F[B.Foff + (int64_t)k * RR + q] : 0.f;
}

// Phase 2 on the term-contiguous copy: 4 * NQ terms per thread, read as NQ float4 per translate.
// Phase 2 (FP32).  One thread per pixel and 4 NQ terms; a block covers a TX x (256 / TX) pixel
// tile (TX consecutive pixels along axis 1 per block row, so that a warp's dL/ds and F loads are
// contiguous), and blockIdx.x = tile column * zc + term group: the zc blocks of a tile are
// adjacent in launch order, so that they run together and share the tile's dL/ds reads through L2.
template <int NQ, int TX>
__global__ void __launch_bounds__(256) k_bwd_dv4(const __grid_constant__ BwdDev bd, const float* __restrict__ FT,
                                                 const float* __restrict__ S, float* __restrict__ dv)
{
    const int n = bd.n;
    const int zc = (bd.m + 4 * NQ - 1) / (4 * NQ);
    const int tx = blockIdx.x / zc;
    const int kbase = (blockIdx.x - tx * zc) * 4 * NQ;
    const int x0 = blockIdx.y * (256 / TX) + threadIdx.y, x1 = tx * TX + threadIdx.x;
    if (x0 >= n || x1 >= n) return;
    float4 acc[NQ];
#pragma unroll
    for (int g = 0; g < NQ; ++g) acc[g] = make_float4(0.f, 0.f, 0.f, 0.f);
    const int ng = min(NQ, (bd.mp - kbase) >> 2);  // float4 groups present in the copy
    for (int b = 0; b < bd.nb; ++b) {
        const BwdBand& B = bd.band[b];
        const int lg = B.j, njm = B.nj - 1;
        const int a0 = x0 - B.P0, a1 = x1 - B.P1;
        const int l0lo = -((-(a0 - B.R0 + 1)) >> lg), l0hi = a0 >> lg;
        const int l1lo = -((-(a1 - B.R1 + 1)) >> lg), l1hi = a1 >> lg;
        const int RR = B.R0 * B.R1;
        const float4* Fa = reinterpret_cast<const float4*>(FT + B.FToff) + (int64_t)(kbase >> 2) * RR;
        const float* Sb = S + B.Soff;
        for (int l0 = l0lo; l0 <= l0hi; ++l0) {
            const int q0 = a0 - (l0 << lg);
            const int64_t rb = (int64_t)(l0 & njm) * B.nj;
#pragma unroll 2
            for (int l1 = l1lo; l1 <= l1hi; ++l1) {
                const int q = q0 * B.R1 + (a1 - (l1 << lg));
                const float sv = __ldg(Sb + (rb + (l1 & njm)) * RR + q);
#pragma unroll
                for (int g = 0; g < NQ; ++g) {
                    if (g < ng) {
                        const float4 f = __ldg(Fa + (int64_t)g * RR + q);
                        acc[g].x = fmaf(f.x, sv, acc[g].x);
                        acc[g].y = fmaf(f.y, sv, acc[g].y);
                        acc[g].z = fmaf(f.z, sv, acc[g].z);
                        acc[g].w = fmaf(f.w, sv, acc[g].w);
                    }
                }
            }
        }
    }
    const int64_t pix = (int64_t)x0 * n + x1;
#pragma unroll
    for (int g = 0; g < NQ; ++g) {
        const float r[4] = {acc[g].x, acc[g].y, acc[g].z, acc[g].w};
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (kbase + 4 * g + k < bd.m) dv[(int64_t)(kbase + 4 * g + k) * bd.N + pix] = r[k];
    }
}

// Phase 2.  One thread per pixel (16 x 16 tiles) and KC terms (blockIdx.z picks the chunk);
// the translate loop is unrolled by 2 so that loads of consecutive translates overlap.
template <typename T, int KC>
__global__ void __launch_bounds__(256) k_bwd_dv(const __grid_constant__ BwdDev bd, const T* __restrict__ F,
                                                const T* __restrict__ S, T* __restrict__ dv)
{
    const int n = bd.n;
    const int kbase = blockIdx.z * KC;
    const int x0 = blockIdx.y * 16 + threadIdx.y, x1 = blockIdx.x * 16 + threadIdx.x;
    if (x0 >= n || x1 >= n) return;
    T acc[KC];
#pragma unroll
    for (int k = 0; k < KC; ++k) acc[k] = T(0);
    const int kn = min(KC, bd.m - kbase);
    for (int b = 0; b < bd.nb; ++b) {
        const BwdBand& B = bd.band[b];
        const int lg = B.j, njm = B.nj - 1;
        // unwrapped translates whose region [2^j l + P, + R) contains x (mod n)
        const int a0 = x0 - B.P0, a1 = x1 - B.P1;
        const int l0lo = -((-(a0 - B.R0 + 1)) >> lg), l0hi = a0 >> lg;
        const int l1lo = -((-(a1 - B.R1 + 1)) >> lg), l1hi = a1 >> lg;
        const int RR = B.R0 * B.R1;
        const T* Fb = F + B.Foff + (int64_t)kbase * RR;
        const T* Sb = S + B.Soff;
        for (int l0 = l0lo; l0 <= l0hi; ++l0) {
            const int q0 = a0 - (l0 << lg);
            const int64_t rb = (int64_t)(l0 & njm) * B.nj;
            int l1 = l1lo;
            for (; l1 + 1 <= l1hi; l1 += 2) {
                const int qa = q0 * B.R1 + (a1 - (l1 << lg)), qb = qa - (1 << lg);
                const T sa = __ldg(Sb + (rb + (l1 & njm)) * RR + qa);
                const T sb = __ldg(Sb + (rb + ((l1 + 1) & njm)) * RR + qb);
#pragma unroll
                for (int k = 0; k < KC; ++k)
                    if (k < kn)
                        acc[k] = fma(__ldg(Fb + (int64_t)k * RR + qb), sb,
                                     fma(__ldg(Fb + (int64_t)k * RR + qa), sa, acc[k]));
            }
            if (l1 <= l1hi) {
                const int qa = q0 * B.R1 + (a1 - (l1 << lg));
                const T sa = __ldg(Sb + (rb + (l1 & njm)) * RR + qa);
#pragma unroll
                for (int k = 0; k < KC; ++k)
                    if (k < kn) acc[k] = fma(__ldg(Fb + (int64_t)k * RR + qa), sa, acc[k]);
            }
        }
    }
    const int64_t pix = (int64_t)x0 * n + x1;
#pragma unroll
    for (int k = 0; k < KC; ++k)
        if (k < kn) dv[(int64_t)(kbase + k) * bd.N + pix] = acc[k];
}

// Phase 3.  Block (band, 128 region positions, chunk of rows); KC terms per block (blockIdx.z).
// Only the terms whose window is nonzero on a row's region (the row's active mask, written by
// phase 1) are read.
template <typename T, int KC>
__global__ void __launch_bounds__(128) k_bwd_dF(const __grid_constant__ BwdDev bd, const T* __restrict__ v,
                                                const T* __restrict__ S, const unsigned long long* __restrict__ amask,
                                                int mwords, T* __restrict__ dF, const int* __restrict__ blk_off,
                                                int chunk)
{
    // blockIdx.x enumerates (band, region block of 128, chunk of rows) over all bands
    int b = 0;
    while (b + 1 < bd.nb && (int)blockIdx.x >= blk_off[b + 1]) ++b;
    const BwdBand& B = bd.band[b];
    const int bl = blockIdx.x - blk_off[b];
    const int qblocks = (B.R0 * B.R1 + 127) / 128;
    const int qb = bl % qblocks, cb = bl / qblocks;
    const int RR = B.R0 * B.R1;
    const int q = qb * 128 + threadIdx.x;
    if (q >= RR) return;
    const int kbase = blockIdx.z * KC;
    const int n = bd.n, lg = B.j;
    const int q0 = q / B.R1, q1 = q - q0 * B.R1;
    const int rows = B.nj * B.nj;
    const int rbeg = cb * chunk, rend = min(rows, rbeg + chunk);
    T acc[KC];
#pragma unroll
    for (int k = 0; k < KC; ++k) acc[k] = T(0);
    const int lgn = log2i(B.nj);
#pragma unroll 4
    for (int rl = rbeg; rl < rend; ++rl) {
        const int l0 = rl >> lgn, l1 = rl & (B.nj - 1);
        const int gy = ((l0 << lg) + B.P0 + q0) & (n - 1), gx = ((l1 << lg) + B.P1 + q1) & (n - 1);
        const int64_t pix = (int64_t)gy * n + gx;
        const T s = __ldg(S + B.Soff + (int64_t)rl * RR + q);
        const unsigned long long mk = __ldg(amask + (B.rowoff + rl) * mwords + (kbase >> 6)) >> (kbase & 63);
#pragma unroll
        for (int k = 0; k < KC; ++k)
            if ((mk >> k) & 1ull) acc[k] = fma(__ldg(v + (int64_t)(kbase + k) * bd.N + pix), s, acc[k]);
    }
    const int kn = min(KC, bd.m - kbase);
#pragma unroll
    for (int k = 0; k < KC; ++k)
        if (k < kn) atomicAdd(dF + B.Foff + (int64_t)(kbase + k) * RR + q, acc[k]);
}

// Phase 3 with the per-pixel window lists: the same blocks as k_bwd_dF, but a region position
// visits only the (at most `slots`) windows nonzero at its pixel; each thread keeps the m
// partial sums of its position in its own column of shared memory ([m][128]).
// Rows of one dL/dF block at one region position q: for each row, the dL/ds value and the NS
// window-list slots of its pixel, accumulated into the thread's column of acc (acc[k * 128]).
template <typename T, int NS>
__device__ __forceinline__ void dF_rows(const WSlot<T>* __restrict__ wl, int N, const T* __restrict__ Sq, int RR,
                                        int rbeg, int rend, int lgn, int njm, int lg, int p0, int p1, int nm, int n,
                                        T* acc)
{
#pragma unroll 2
    for (int rl = rbeg; rl < rend; ++rl) {
        const int l0 = rl >> lgn, l1 = rl & njm;
        const int pix = (((l0 << lg) + p0) & nm) * n + (((l1 << lg) + p1) & nm);
        const T sv = __ldg(Sq + (int64_t)rl * RR);
        WSlot<T> w[NS];
#pragma unroll
        for (int sl = 0; sl < NS; ++sl) w[sl] = load_slot(wl + (pix + sl * N));
#pragma unroll
        for (int sl = 0; sl < NS; ++sl)
            if (w[sl].v != T(0)) acc[(int)w[sl].k * 128] += w[sl].v * sv;
    }
}

template <typename T>
__global__ void __launch_bounds__(128) k_bwd_dF_wl(const __grid_constant__ BwdDev bd, const WSlot<T>* __restrict__ wl,
                                                   int slots, const T* __restrict__ S, T* __restrict__ dF,
                                                   const int* __restrict__ blk_off, int chunk)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* acc = reinterpret_cast<T*>(smem_raw) + threadIdx.x;  // acc[k * 128]
    int b = 0;
    while (b + 1 < bd.nb && (int)blockIdx.x >= blk_off[b + 1]) ++b;
    const BwdBand& B = bd.band[b];
    const int bl = blockIdx.x - blk_off[b];
    const int qblocks = (B.R0 * B.R1 + 127) / 128;
    const int qb = bl % qblocks, cb = bl / qblocks;
    const int RR = B.R0 * B.R1;
    const int q = qb * 128 + threadIdx.x;
    if (q >= RR) return;
    const int n = bd.n, lg = B.j, m = bd.m;
    const int N = (int)bd.N;
    for (int k = 0; k < m; ++k) acc[k * 128] = T(0);
    const int q0 = q / B.R1, q1 = q - q0 * B.R1;
    const int rows = B.nj * B.nj;
    const int rbeg = cb * chunk, rend = min(rows, rbeg + chunk);
    const int lgn = log2i(B.nj);
    const T* Sq = S + B.Soff + q;  // row rl's value at + rl * RR
    const int p0 = B.P0 + q0, p1 = B.P1 + q1, nm = n - 1, njm = B.nj - 1;
    switch (slots) {
        case 1: dF_rows<T, 1>(wl, N, Sq, RR, rbeg, rend, lgn, njm, lg, p0, p1, nm, n, acc); break;
        case 2: dF_rows<T, 2>(wl, N, Sq, RR, rbeg, rend, lgn, njm, lg, p0, p1, nm, n, acc); break;
        case 3: dF_rows<T, 3>(wl, N, Sq, RR, rbeg, rend, lgn, njm, lg, p0, p1, nm, n, acc); break;
        case 4: dF_rows<T, 4>(wl, N, Sq, RR, rbeg, rend, lgn, njm, lg, p0, p1, nm, n, acc); break;
        default:
            for (int rl = rbeg; rl < rend; ++rl) {
                const int l0 = rl >> lgn, l1 = rl & njm;
                const int pix = (((l0 << lg) + p0) & nm) * n + (((l1 << lg) + p1) & nm);
                const T sv = __ldg(Sq + (int64_t)rl * RR);
                for (int sl = 0; sl < slots; ++sl) {
                    const WSlot<T> w = load_slot(wl + (pix + sl * N));
                    if (w.v != T(0)) acc[(int)w.k * 128] += w.v * sv;
                }
            }
    }
    for (int k = 0; k < m; ++k) {
        const T a = acc[k * 128];
        if (a != T(0)) atomicAdd(dF + B.Foff + (int64_t)k * RR + q, a);
    }
}

}  // namespace pcw
