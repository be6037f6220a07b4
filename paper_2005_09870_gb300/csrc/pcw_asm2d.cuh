// 2-D row assembly and its adjoint, register-blocked.
//
// Stage 1 (k_s_tiles, one launch over all rows): s(q) = sum_k v_k(g + q) F_{k,b}(q) over the
// windows nonzero at each pixel, compensated over k (FP32), into the s scratch.
// Stage 2, one stored row per thread group (gt threads; several groups per CTA): the row's s,
//   level 1 (or LL of level k0 by the scaling filter phi_{k0} at stride 2^k0 for rows whose
//   finest kept level is k0 + 1), then the cascade on LL up to the coarsest kept level; the
//   coefficients inside the row's stencil windows are written to its storage segment.
// The low/high-pass passes hold a sliding window of 2*CH + 2*LF - 4 inputs in registers and
// produce CH low-pass and CH high-pass outputs per work item (taps unrolled, LF = filter
// length as a template parameter; shorter filters run zero-padded).
#pragma once
#include <type_traits>

#include "pcw_kernels.cuh"

namespace pcw {


template <typename T>
__device__ __forceinline__ void kahan_add(T& s, T& c, T x)
{
    s += x;
}
template <>
__device__ __forceinline__ void kahan_add<float>(float& s, float& c, float x)
{
    const float y = __fsub_rn(x, c);
    const float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
}

// floor(x / w) for 0 <= x < 2^21 and 1 <= w < 2^24, from a reciprocal of w: (x + 1/2) / w lies at
// least 1/(2w) from an integer, and the float product errs by under 2^-21 (x + 1/2) / w.
__device__ __forceinline__ int div_small(int x, float inv_w) { return __float2int_rz(((float)x + 0.5f) * inv_w); }

// Steps (a, b) through a row-major count x W grid by gt per iteration (no divisions).
struct Stepper {
    int a, b, da, db, W;
    __device__ __forceinline__ void init(int start, int step, int w)
    {
        W = w;
        const float inv = 1.0f / (float)w;
        a = div_small(start, inv);
        b = start - a * w;
        da = div_small(step, inv);
        db = step - da * w;
    }
    __device__ __forceinline__ void next()
    {
        a += da;
        b += db;
        if (b >= W) {
            b -= W;
            ++a;
        }
    }
};

// Zeroes the margins of a padded array: [0, lead) and the pitch - len elements after each of
// its nl lines (line l at lead + l * pitch).  One line's gap (or the lead) per thread, as up to
// GMAX >= max(lead, pitch - len) unrolled stores.
template <typename T, int GMAX>
__device__ __forceinline__ void zero_gaps(T* a, int lead, int nl, int len, int pitch, int tid, int gt)
{
    const int g = pitch - len;
    for (int l = tid; l <= nl; l += gt) {
        T* p = (l < nl) ? a + lead + l * pitch + len : a;
        const int cnt = (l < nl) ? g : lead;
#pragma unroll
        for (int i = 0; i < GMAX; ++i)
            if (i < cnt) p[i] = T(0);
    }
}

// Low/high-pass pass along one axis over nlines contiguous input lines (line l starts at
// in + l * lstride).  Low-pass output c of line l goes to outL[l + c * osL], high-pass output to
// outH[l + c * osH]: the result is stored transposed, so the next pass again reads contiguous
// lines.  Output c (unwrapped ro.lo + c) reads inputs 2(ro.lo + c) + [2 - LF, LF - 1].  Unless
// the output range wraps, the input is a padded array (zero margins, see pass_margin) and the
// window loads carry no bounds checks.
template <typename T, int LF, int CH>
__device__ __forceinline__ void pass_hg(const T* in, int lstride, Range ri, int n_in, T* outL, int osL, T* outH,
                                        int osH, Range ro, int nlines, const T (&hr)[LF], const T (&gr)[LF], int tid,
                                        int gt)
{
    constexpr int WN = 2 * CH + 2 * LF - 4;
    const int nch = (ro.cnt + CH - 1) / CH;
    const int items = nlines * nch;
    Stepper st;  // a = chunk, b = line: consecutive lanes walk lines
    st.init(tid, gt, nlines);
    const int nim = n_in - 1;
    const int base0 = 2 * ro.lo + (2 - LF) - ri.lo;
    for (int it = tid; it < items; it += gt, st.next()) {
        const int line = st.b, c0 = st.a * CH;
        const int base = base0 + 2 * c0;
        const T* src = in + line * lstride;
        T w[WN];
        if (!ro.full) {
#pragma unroll
            for (int i = 0; i < WN; ++i) w[i] = src[base + i];
        } else {
#pragma unroll
            for (int i = 0; i < WN; ++i) {
                const int p = (base + i) & nim;
                w[i] = (p < ri.cnt) ? src[p] : T(0);
            }
        }
        T* oL = outL + line + c0 * osL;
        T* oH = outH + line + c0 * osH;
#pragma unroll
        for (int o = 0; o < CH; ++o) {
            T a = T(0), d = T(0);
#pragma unroll
            for (int i = 0; i < LF; ++i) {
                a = fma(hr[i], w[2 * o + LF - 2 + i], a);
                d = fma(gr[i], w[2 * o + i], d);
            }
            if (c0 + o < ro.cnt) {
                oL[o * osL] = a;
                oH[o * osH] = d;
            }
        }
    }
}

// Low-pass only (scaling filter f of length len at stride S, taps at offsets [0, len)).
template <typename T>
__device__ __forceinline__ void pass_lo(const T* in, int lstride, int stride, Range ri, int n_in, T* out,
                                        int olstride, int ostride, Range ro, int nlines, const T* f, int len, int S,
                                        int tid, int gt)
{
    const int items = nlines * ro.cnt;
    Stepper st;
    st.init(tid, gt, nlines);
    const int nim = n_in - 1;
    for (int it = tid; it < items; it += gt, st.next()) {
        const int line = st.b, c = st.a;
        const T* x = in + line * lstride;
        const int x0 = S * (ro.lo + c) - ri.lo;
        T acc = T(0), acc2 = T(0);
        if (!ro.full) {
            const int ilo = x0 < 0 ? -x0 : 0;
            const int ihi = min(len, ri.cnt - x0);
            int i = ilo;
            for (; i + 1 < ihi; i += 2) {
                acc = fma(f[i], x[(x0 + i) * stride], acc);
                acc2 = fma(f[i + 1], x[(x0 + i + 1) * stride], acc2);
            }
            if (i < ihi) acc = fma(f[i], x[(x0 + i) * stride], acc);
        } else {
            for (int i = 0; i < len; ++i) {
                const int p = (x0 + i) & nim;
                if (p < ri.cnt) acc = fma(f[i], x[p * stride], acc);
            }
        }
        out[line * olstride + c * ostride] = acc + acc2;
    }
}


// Position stepping over a W0 x W1 window held in a shared-memory array of row pitch pz, for
// copies between the window and a row's storage (the window row-major and contiguous there).
// A thread takes entries e, e + step, e + 2 step, ... (consecutive entries on consecutive
// threads: coalesced in global memory, free of bank conflicts in shared memory); zi is the
// shared-memory offset of its current entry, advanced without divisions.
struct WinStep {
    int zi, b, dz, db, wrapz, W1;
    __device__ __forceinline__ void init(int e, int step, int pz, int w1)
    {
        W1 = w1;
        const float inv = 1.0f / (float)w1;
        const int a = div_small(e, inv), da = div_small(step, inv);
        b = e - a * w1;
        db = step - da * w1;
        zi = a * pz + b;
        dz = da * pz + db;
        wrapz = pz - w1;
    }
    __device__ __forceinline__ void next()
    {
        b += db;
        zi += dz;
        if (b >= W1) {
            b -= W1;
            zi += wrapz;
        }
    }
};

// Copies the stencil window of one column band from its coefficient array (pitch pz) to the
// row's storage (and the BF16 copy), which holds the window row-major.
template <typename T>
__device__ __forceinline__ void write_win(const OpDev<T>& op, const T* Zb, int pz, Range r0, Range r1, int nj, int f0,
                                          int W0, int f1, int W1, int64_t dst, int tid, int gt)
{
    const int tot = W0 * W1;
    if (tot <= 0) return;
    T* th = op.theta + dst;
    __nv_bfloat16* t16 = op.theta16 ? op.theta16 + dst : nullptr;
    if (!r0.full && !r1.full && op.gap >= 0) {
        const T* z = Zb + (f0 - r0.lo) * pz + (f1 - r1.lo);  // inside the array (checked by the planner)
        WinStep ws;
        ws.init(tid, gt, pz, W1);
        for (int idx = tid; idx < tot; idx += gt) {
            const T val = z[ws.zi];
            th[idx] = val;
            if (t16) t16[idx] = __float2bfloat16_rn((float)val);
            ws.next();
        }
    } else {
        Stepper st;
        st.init(tid, gt, W1);
        for (int idx = tid; idx < tot; idx += gt, st.next()) {
            const int p0 = pmod(f0 + st.a - r0.lo, nj), p1 = pmod(f1 + st.b - r1.lo, nj);
            const bool ok = (r0.full || p0 < r0.cnt) && (r1.full || p1 < r1.cnt);
            const T val = ok ? Zb[p0 * pz + p1] : T(0);
            th[idx] = val;
            if (t16) t16[idx] = __float2bfloat16_rn((float)val);
        }
    }
}

// Stage 1 of every stored 2-D row in one launch: s(q) = sum over the window list of pixel
// g + q of v_k * F_{k,b}(q) (the windows nonzero there, in increasing k), compensated,
// written to op.sf + Soff[b] + rl * RR + q.  One warp per stored row (canonical order, eight
// rows per CTA); its lanes walk the region positions.  Indices are 32-bit: a region, a
// window list (slots x N) and a band's F stay far below 2^31 elements.
// Tiles of the window sums: T consecutive rows of one band along axis 1 (same l0).  Their
// regions, shifted by 2^j from row to row, cover a union of R0 x (R1 + (T - 1) 2^j) pixels
// (axis 1 unwrapped: a pixel the union meets twice counts twice); a block walks the union once,
// loads each pixel's window list once and produces s for every row of the tile whose region
// holds the pixel.
struct STiles {
    int T;                    // rows per tile along axis 1
    int tile_off[MAXB + 1];   // first tile of each band (bands in canonical order)
};

// s of the rows t in [t_lo, t_hi] of a tile at one union pixel, with NS window-list slots: the
// slots are loaded once, then for each row its F values (all loads first) and the compensated
// sum over the slots.
template <typename T, int NS>
__device__ __forceinline__ void s_tile_pixel(const WSlot<T>* __restrict__ wp, int N, const T* __restrict__ F0, int RR,
                                             int qbase, int sq, int t_lo, int t_hi, T* __restrict__ out)
{
    WSlot<T> w[NS];
#pragma unroll
    for (int sl = 0; sl < NS; ++sl) w[sl] = load_slot(wp + sl * N);
    for (int t = t_lo; t <= t_hi; ++t) {
        const int q = qbase - t * sq;  // position in row t's region
        T f[NS];
#pragma unroll
        for (int sl = 0; sl < NS; ++sl) f[sl] = __ldg(F0 + ((int)w[sl].k * RR + q));
        T acc = w[0].v * f[0], c = T(0);
#pragma unroll
        for (int sl = 1; sl < NS; ++sl) kahan_add(acc, c, w[sl].v * f[sl]);
        out[(int64_t)t * RR + q] = acc;
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_s_tiles(const OpDev<T>* __restrict__ opd, const __grid_constant__ STiles tl)
{
    __shared__ int b_s;
    const OpDev<T>& op = *opd;  // device copy (refreshed before each run, also inside graphs)
    const int n = op.n, nm = n - 1, nb = op.nb;
    if (threadIdx.x < 32) {
        // band of the tile: the last band whose first tile is at or before it
        const int lane = threadIdx.x;
        const unsigned m1 = __ballot_sync(0xffffffffu, lane < nb && tl.tile_off[lane] <= (int)blockIdx.x);
        const unsigned m2 =
            __ballot_sync(0xffffffffu, lane + 32 < nb && tl.tile_off[min(lane + 32, MAXB)] <= (int)blockIdx.x);
        if (lane == 0) b_s = m2 ? 63 - __clz(m2) : 31 - __clz(m1);
    }
    __syncthreads();
    const int b = b_s;
    const Band Bo = band_info(2, n, op.L, b);
    const int nt1 = (Bo.nj + tl.T - 1) / tl.T;
    const int tb = blockIdx.x - tl.tile_off[b];
    const int l0 = tb / nt1, l1s = (tb - l0 * nt1) * tl.T;
    const int nr = min(tl.T, Bo.nj - l1s);
    const Range R0 = region0(Bo.j, Bo.e0, l0, op.r, op.Lf, n);
    const Range R1 = region0(Bo.j, Bo.e1, l1s, op.r, op.Lf, n);  // the tile's first row
    const int lg = Bo.j, sq = 1 << lg;
    const int c1 = R1.cnt, RR = R0.cnt * c1;
    const bool full1 = R1.full;
    const int U1 = full1 ? n : c1 + (nr - 1) * sq;
    const int g0 = pmod(R0.lo, n), g1 = pmod(R1.lo, n);
    const T* F0 = op.F + op.Foff[b];
    T* out = op.sf + op.Soff[b] + ((int64_t)l0 * Bo.nj + l1s) * RR;
    const WSlot<T>* wl = reinterpret_cast<const WSlot<T>*>(op.wl);
    const int S = op.wl_slots, N = (int)op.N;
    const int tot = R0.cnt * U1;
    const float inv = 1.0f / (float)U1;
    int a = div_small(threadIdx.x, inv), c = threadIdx.x - a * U1;
    const int da = div_small(blockDim.x, inv), dc = blockDim.x - da * U1;
    for (int e = threadIdx.x; e < tot; e += blockDim.x) {
        const int pix = ((g0 + a) & nm) * n + ((g1 + c) & nm);
        // rows of the tile whose region holds union column c: c - t 2^j in [0, c1)
        int t_lo, t_hi, qbase;
        if (full1) {
            // every row covers every pixel; row t's column is (c - t 2^j) mod n, handled row by row
            for (int t = 0; t < nr; ++t) {
                const int q = a * c1 + ((c - t * sq) & nm);
                T acc = T(0), cc = T(0);
                for (int sl = 0; sl < S; ++sl) {
                    const WSlot<T> w = load_slot(wl + (pix + sl * N));
                    if (w.v != T(0)) kahan_add(acc, cc, w.v * __ldg(F0 + ((int)w.k * RR + q)));
                }
                out[(int64_t)t * RR + q] = acc;
            }
        } else {
            t_lo = max(0, -((-(c - c1 + 1)) >> lg));
            t_hi = min(nr - 1, c >> lg);
            qbase = a * c1 + c;
            const WSlot<T>* wp = wl + pix;
            switch (S) {
                case 1: s_tile_pixel<T, 1>(wp, N, F0, RR, qbase, sq, t_lo, t_hi, out); break;
                case 2: s_tile_pixel<T, 2>(wp, N, F0, RR, qbase, sq, t_lo, t_hi, out); break;
                case 3: s_tile_pixel<T, 3>(wp, N, F0, RR, qbase, sq, t_lo, t_hi, out); break;
                case 4: s_tile_pixel<T, 4>(wp, N, F0, RR, qbase, sq, t_lo, t_hi, out); break;
                default:
                    for (int t = t_lo; t <= t_hi; ++t) {
                        const int q = qbase - t * sq;
                        T acc = T(0), cc = T(0);
                        for (int sl = 0; sl < S; ++sl) {
                            const WSlot<T> w = load_slot(wp + sl * N);
                            if (w.v != T(0)) kahan_add(acc, cc, w.v * __ldg(F0 + ((int)w.k * RR + q)));
                        }
                        out[(int64_t)t * RR + q] = acc;
                    }
            }
        }
        a += da;
        c += dc;
        if (c >= U1) {
            c -= U1;
            ++a;
        }
    }
}

// Per-row constants of a 2-D row.
struct Row2 {
    Band Bo;
    int j, jlo, jhi, k0, l0, l1, g0, g1;
    Range A0, A1;
    int64_t srow, row_base;
};

template <typename T>
__device__ __forceinline__ Row2 row2_setup(const OpDev<T>& op, int b, int rl)
{
    Row2 R;
    const int n = op.n, L = op.L;
    const int dense = op.gap < 0;
    R.Bo = band_info(2, n, L, b);
    R.j = R.Bo.j;
    R.jlo = dense ? 1 : max(1, R.j - op.gap);
    R.jhi = dense ? L : min(L, R.j + op.gap);
    R.k0 = R.jlo - 1;
    const int lg = log2i(R.Bo.nj);
    R.l0 = rl >> lg;
    R.l1 = rl & (R.Bo.nj - 1);
    R.A0 = region0(R.j, R.Bo.e0, R.l0, op.r, op.Lf, n);
    R.A1 = region0(R.j, R.Bo.e1, R.l1, op.r, op.Lf, n);
    R.g0 = pmod(R.A0.lo, n);
    R.g1 = pmod(R.A1.lo, n);
    R.srow = R.Bo.off + rl;
    R.row_base = op.row_ptr[R.srow];
    return R;
}

// Block offsets and the active term list of a row (meta area of its group), computed by the
// group's first warp with lane-parallel counts and warp scans.  Ends with a group barrier;
// returns false (uniformly) when the row length disagrees with row_ptr.
template <typename T>
__device__ __forceinline__ bool row2_meta(const OpDev<T>& op, const Row2& R, int b, int* meta, int tid, int gt,
                                          int gid, bool terms)
{
    const int n = op.n, L = op.L;
    const int lane = threadIdx.x & 31;
    if (tid < 32) {
        // OR of the tile masks over the region (only when the active-term list is wanted)
        unsigned long long mw[MAXW];
#pragma unroll
        for (int w = 0; w < MAXW; ++w) mw[w] = 0ull;
        const int ts0 = op.ts0, ts1 = op.ts1;
        const int s0 = terms ? R.g0 / ts0 : 0, s1 = terms ? R.g1 / ts1 : 0;
        const int nt0 = terms ? min(op.tpa0, (R.g0 % ts0 + R.A0.cnt + ts0 - 1) / ts0) : 0;
        const int nt1 = terms ? min(op.tpa1, (R.g1 % ts1 + R.A1.cnt + ts1 - 1) / ts1) : 0;
        for (int i = lane; i < nt0 * nt1; i += 32) {
            const int i0 = i / nt1;
            const int t0 = (s0 + i0) % op.tpa0, t1 = (s1 + i - i0 * nt1) % op.tpa1;
            const unsigned long long* mp = op.masks + ((int64_t)t0 * op.tpa1 + t1) * op.mwords;
#pragma unroll
            for (int w = 0; w < MAXW; ++w)
                if (w < op.mwords) mw[w] |= mp[w];
        }
        // stencil windows and block counts: lane b2 (and b2 + 32); exclusive scan of the counts
        // in canonical band order
        int total = 0;
        const int dense = op.gap < 0;
        for (int base = 0; base < op.nb; base += 32) {
            const int b2 = base + lane;
            int cnt = 0;
            if (b2 < op.nb && block_kept(2, n, L, op.gap, b, b2)) {
                const Band B2 = band_info(2, n, L, b2);
                int f0, W0, f1, W1;
                stencil(R.j, R.Bo.e0, R.l0, B2.j, B2.e0, op.r, op.Lf, n, dense, &f0, &W0);
                stencil(R.j, R.Bo.e1, R.l1, B2.j, B2.e1, op.r, op.Lf, n, dense, &f1, &W1);
                int* w = meta + WIN_OFF + 4 * b2;
                w[0] = f0;
                w[1] = W0;
                w[2] = f1;
                w[3] = W1;
                cnt = W0 * W1;
            }
            int x = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            if (b2 < op.nb) meta[b2] = total + x - cnt;
            total += __shfl_sync(0xffffffffu, x, 31);
        }
        // active terms: ballot over the OR-reduced mask bits
        unsigned char* act = reinterpret_cast<unsigned char*>(meta + ACT_OFF);
        int na = 0;
#pragma unroll
        for (int w = 0; w < MAXW; ++w) {
            if (w >= op.mwords || !terms) break;
            const unsigned lo = __reduce_or_sync(0xffffffffu, (unsigned)mw[w]);
            const unsigned hi = __reduce_or_sync(0xffffffffu, (unsigned)(mw[w] >> 32));
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                const unsigned word = half ? hi : lo;
                const bool bit = (word >> lane) & 1u;
                const unsigned ball = __ballot_sync(0xffffffffu, bit);
                if (bit) act[na + __popc(ball & ((1u << lane) - 1u))] = (unsigned char)(w * 64 + half * 32 + lane);
                na += __popc(ball);
            }
        }
        if (lane == 0) {
            meta[op.nb] = total;
            meta[NACT_OFF] = na;
            if ((int64_t)total != op.row_ptr[R.srow + 1] - R.row_base) flag_error(op.err, ERR_ROWLEN);
        }
    }
    group_sync(gt, gid);
    return (int64_t)meta[op.nb] == op.row_ptr[R.srow + 1] - R.row_base;
}

// Writes the three detail bands of level jj (and the approximation band when jj == L):
// D = [(0,1) | (1,0) | (1,1)], each q0r.cnt x q1r.cnt at pitch q1r.cnt; LL at pitch LP.
template <typename T>
__device__ __forceinline__ void write_level(const OpDev<T>& op, const Row2& R, const int* meta, const T* LL, int LP,
                                            const T* D, Range q0r, Range q1r, int jj, int tid, int gt)
{
    const int n = op.n, L = op.L, dense = op.gap < 0;
    const int dq = q0r.cnt * q1r.cnt, nj = n >> jj;
    const int tmax = (jj == L) ? 4 : 3;
    for (int t = 0; t < tmax; ++t) {
        const int b2 = (t == 3) ? 0 : band_of_level(2, L, jj, t);
        const int e0 = (t == 3) ? 0 : (t >= 1 ? 1 : 0), e1 = (t == 3) ? 0 : (t == 1 ? 0 : 1);
        (void)e0;
        (void)e1;
        (void)dense;
        const int* w = meta + WIN_OFF + 4 * b2;
        const int f0 = w[0], W0 = w[1], f1 = w[2], W1 = w[3];
        write_win(op, (t == 3) ? LL : D + t * dq, (t == 3) ? LP : q1r.cnt, q0r, q1r, nj, f0, W0, f1, W1,
                  R.row_base + meta[b2], tid, gt);
    }
}

// Filter area of a 2-D row kernel for rows of band b: h padded to LF | g right-aligned in LF
// (tap i at position 2 - LF + i) | phi_{k0} when the band's first produced level is k0 > 0.
template <typename T, int LF>
__device__ __forceinline__ void load_filters2d(const OpDev<T>& op, int b, T* fS)
{
    const int Lf = op.Lf;
    const Band Bo = band_info(2, op.n, op.L, b);
    const int jlo = (op.gap < 0) ? 1 : max(1, Bo.j - op.gap);
    const int k0 = jlo - 1;
    const int lenk = (k0 > 0) ? wav_len(k0, Lf) : 0;
    for (int i = threadIdx.x; i < LF; i += blockDim.x) {
        fS[i] = (i < Lf) ? op.taps[i] : T(0);
        fS[LF + i] = (i >= LF - Lf) ? op.taps[Lf + i - (LF - Lf)] : T(0);
    }
    for (int i = threadIdx.x; i < lenk; i += blockDim.x) fS[2 * LF + i] = op.wav[op.wofs[k0] + i];
}

// One stored 2-D row (band cfg.b, translate index rl) by one thread group.
template <typename T, int LF>
__device__ __forceinline__ void asm2d_row(const OpDev<T>& op, const AsmCfg& cfg, int rl, const T* fS, int* meta,
                                          T* arena, int gid, int tid)
{
    constexpr int CH = PASS_CH;
    const int gt = cfg.gt;
    const int n = op.n, Lf = op.Lf;
    T* const arena_end = arena + cfg.arena;
    const int A = cfg.arena;
    const Row2 R = row2_setup(op, cfg.b, rl);
    if (!row2_meta(op, R, cfg.b, meta, tid, gt, gid, false)) return;  // s comes from k_s_tiles: no term list
    const int k0 = R.k0;
    const int lenk = (k0 > 0) ? wav_len(k0, Lf) : 0;

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

    // Level loop.  The first produced level is 1 (cascade step on s), or k0 when the row's
    // finest kept level is k0 + 1 > 1 (LL of level k0 directly by phi_k0 at stride 2^k0).
    // Arena: the level's input lines (s rows, or LL of the previous level) and its outputs
    // (LL, then the detail bands) at the start, the axis-1 results Y at the end.  Every array a
    // low/high-pass pass reads is padded (pass_margin): s rows at pitch XP, Y transposed (one
    // line per axis-1 coefficient), LL at pitch LP.
    const int mg = pass_margin(Lf, LF);
    const int XP = (k0 > 0) ? (A1.cnt | 1) : odd_pitch(A1.cnt, mg);  // the scaling-filter pass checks bounds
    const int lv0 = (k0 == 0) ? 1 : k0;
    Range p0 = A0, p1 = A1;
    T* const xs0 = (k0 > 0) ? arena : arena + mg;  // s rows
    const T* xin = xs0;
    int xpitch = XP;
    int n_in = n;
    int prevZ = 0;
    for (int jj = lv0; jj <= R.jhi; ++jj) {
        const bool first = (jj == lv0);
        const bool lo_only = first && k0 > 0;
        const int nj = n >> jj;
        const int S = lo_only ? (1 << k0) : 2;
        const Range q0r = lo_only ? range_filter(A0, S, 0, lenk, nj) : range_cascade(p0, Lf, nj);
        const Range q1r = lo_only ? range_filter(A1, S, 0, lenk, nj) : range_cascade(p1, Lf, nj);
        const int YP = odd_pitch(p0.cnt, mg);
        const int y1 = lo_only ? p0.cnt * q1r.cnt : padded_size(q1r.cnt, p0.cnt, mg);
        const int ysz = (lo_only ? 1 : 2) * y1;
        const int LP = odd_pitch(q1r.cnt, mg);
        const int llsz = padded_size(q0r.cnt, q1r.cnt, mg);
        const int dq = q0r.cnt * q1r.cnt;
        const int zsz = llsz + (lo_only ? 0 : 3 * dq);
        const int xsz = first ? (lo_only ? B * XP : padded_size(B, A1.cnt, mg)) : prevZ;
        if (xsz + ysz > A || zsz + ysz > A) {
            flag_error(op.err, ERR_ARENA);
            return;
        }
        T* Yl = arena_end - ysz;
        T* Yh = Yl + y1;
        // axis 1 (batched over pixel rows of s on the first level)
        const int nbatch = first ? (A0.cnt + B - 1) / B : 1;
        for (int bi = 0; bi < nbatch; ++bi) {
            const int r0 = bi * B;
            const int nr = first ? min(B, A0.cnt - r0) : p0.cnt;
            if (first) {
                if (bi == 0 && !lo_only) zero_gaps<T, 2 * LF - 2>(arena, mg, B, A1.cnt, XP, tid, gt);
                // s rows computed for all rows beforehand (k_s_tiles), copied asynchronously
                // (cp.async: no register round trip, every copy of the thread in flight at once)
                const T* sr = op.sf + op.Soff[cfg.b] + (int64_t)rl * RR + r0 * A1.cnt;
                const int tot = nr * A1.cnt;
                const float inv = 1.0f / (float)A1.cnt;
                int qa = div_small(tid, inv), qb = tid - qa * A1.cnt;
                const int da = div_small(gt, inv), db = gt - da * A1.cnt;
                for (int e = tid; e < tot; e += gt) {
                    const unsigned dst = (unsigned)__cvta_generic_to_shared(xs0 + qa * XP + qb);
                    if constexpr (sizeof(T) == 4)
                        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(sr + e) : "memory");
                    else
                        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(sr + e) : "memory");
                    qa += da;
                    qb += db;
                    if (qb >= A1.cnt) {
                        qb -= A1.cnt;
                        ++qa;
                    }
                }
                asm volatile("cp.async.wait_all;" ::: "memory");
                group_sync(gt, gid);
            }
            if (lo_only) {
                pass_lo<T>(xs0, XP, 1, A1, n, Yl + r0 * q1r.cnt, q1r.cnt, 1, q1r, nr, phiS, lenk, S, tid, gt);
            } else {
                if (bi == 0) {
                    zero_gaps<T, 2 * LF - 2>(Yl, mg, q1r.cnt, p0.cnt, YP, tid, gt);
                    zero_gaps<T, 2 * LF - 2>(Yh, mg, q1r.cnt, p0.cnt, YP, tid, gt);
                }
                pass_hg<T, LF, CH>(xin, xpitch, p1, n_in, Yl + mg + r0, YP, Yh + mg + r0, YP, q1r, nr, hr, gr, tid,
                                   gt);
            }
            group_sync(gt, gid);
        }
        // axis 0: lines are the axis-1 coefficients (rows of Y^T)
        T* LL = arena + mg;
        T* D = arena + llsz;
        zero_gaps<T, 2 * LF - 2>(arena, mg, q0r.cnt, q1r.cnt, LP, tid, gt);
        if (lo_only) {
            pass_lo<T>(Yl, 1, q1r.cnt, A0, n, LL, 1, LP, q0r, q1r.cnt, phiS, lenk, S, tid, gt);
        } else {
            pass_hg<T, LF, CH>(Yl + mg, YP, p0, n_in, LL, LP, D + dq, q1r.cnt, q0r, q1r.cnt, hr, gr, tid, gt);
            pass_hg<T, LF, CH>(Yh + mg, YP, p0, n_in, D, q1r.cnt, D + 2 * dq, q1r.cnt, q0r, q1r.cnt, hr, gr, tid, gt);
        }
        group_sync(gt, gid);
        if (!lo_only) write_level(op, R, meta, LL, LP, D, q0r, q1r, jj, tid, gt);
        p0 = q0r;
        p1 = q1r;
        xin = LL;
        xpitch = LP;
        n_in = nj;
        prevZ = zsz;
    }
}

template <typename T, int LF>
__global__ void __launch_bounds__(256, 2) k_assemble2d(const __grid_constant__ OpDev<T> op, const AsmCfg cfg)
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
    asm2d_row<T, LF>(op, cfg, cfg.row0 + rloc, fS, meta, arena, gid, tid);
}

// ------------------------------------------------------------------------------------------
// Persistent batched assembly.  Work items (operator, row band, run of rows) are taken
// from a global counter, longest first (the host sorts them).  Each item carries its own
// thread-group shape; the CTA copies the operator's descriptor to shared memory.  FP32.
// ------------------------------------------------------------------------------------------
struct BatchItem {
    int op;   // operator index
    int dim;  // 1 or 2
    int lft;  // 2-D filter template (2, 4, 8 or 20)
    int pad;
    AsmCfg cfg;
};

// KIND selects the row kernel compiled into one instantiation: 1 = 1-D rows, else the 2-D
// filter template LF (2, 4, 8 or 20).  Items of other kinds are not taken: the host queues
// each kind's items in a range of their own with its own counter, so that every instantiation
// holds one row path and keeps its registers.
template <int KIND>
__global__ void __launch_bounds__(256, 2) k_assemble_batch(const OpDev<float>* __restrict__ ops,
                                                           const BatchItem* __restrict__ items, int nitems,
                                                           int* __restrict__ counter)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ OpDev<float> op_s;
    __shared__ BatchItem it_s;
    __shared__ int idx_s;
    for (;;) {
        if (threadIdx.x == 0) idx_s = atomicAdd(counter, 1);
        __syncthreads();
        const int idx = idx_s;
        if (idx >= nitems) return;
        if (threadIdx.x == 0) it_s = items[idx];
        __syncthreads();
        {
            const int* src = reinterpret_cast<const int*>(ops + it_s.op);
            int* dst = reinterpret_cast<int*>(&op_s);
            for (int i = threadIdx.x; i < (int)(sizeof(OpDev<float>) / sizeof(int)); i += blockDim.x) dst[i] = src[i];
        }
        __syncthreads();
        const AsmCfg cfg = it_s.cfg;
        float* fS = reinterpret_cast<float*>(smem_raw);
        if constexpr (KIND == 1) {
            for (int i = threadIdx.x; i < 2 * op_s.Lf; i += blockDim.x) fS[i] = op_s.taps[i];
        } else {
            load_filters2d<float, KIND>(op_s, cfg.b, fS);
        }
        __syncthreads();
        const int gt = cfg.gt;
        const int gid = threadIdx.x / gt, tid = threadIdx.x - gid * gt;
        if (gid < cfg.rpc) {
            int* meta = reinterpret_cast<int*>(smem_raw + sizeof(float) * cfg.filt) + gid * META_INTS;
            float* arena = reinterpret_cast<float*>(smem_raw + sizeof(float) * cfg.filt +
                                                    sizeof(int) * cfg.rpc * META_INTS) +
                           (int64_t)gid * cfg.arena;
            for (int rb = 0; rb < cfg.rows; rb += cfg.rpc) {
                const int rloc = rb + gid;
                if (rloc >= cfg.rows) break;
                const int rl = cfg.row0 + rloc;
                if constexpr (KIND == 1)
                    asm1d_row<float>(op_s, cfg, rl, fS, fS + op_s.Lf, meta, arena, gid, tid);
                else
                    asm2d_row<float, KIND>(op_s, cfg, rl, fS, meta, arena, gid, tid);
                group_sync(gt, gid);  // the group's arena and meta are reused by its next row
            }
        }
        __syncthreads();
    }
}

}  // namespace pcw
