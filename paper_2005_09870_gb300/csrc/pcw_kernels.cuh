// Device kernels of libpcwave (sm_103a).
//
// Pipeline of pc_assemble for one operator (Section 3.2, Algorithm 1 evaluated exactly on
// the prescribed pattern):
//   k_base_wavelets   FP64 cascade of the taps -> phi_{j,0}, psi_{j,0} (Section 2.1)
//   k_filtered_pass1  G = kappa_k (*) rho^{e1}_j along axis 1           } F_{k,beta} = kappa_k * psi_{beta,0},
//   k_filtered_pass2  F = G (*) rho^{e0}_j along axis 0, folded mod n   } the circulant generators of A_k (Lemma 5.1)
//   k_tile_masks      which windows v_k are nonzero on each 16x16 tile
//   k_assemble        per stored row: s = sum_k v_k . F_{k,beta}(. - shift) (compensated over k),
//                     then the localized forward transform of s (Lemma 5.5); its coefficients
//                     inside the stencil are the row's entries of Theta.
// k_apply multiplies the stored matrix by a block of right-hand sides.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "pcw_geom.cuh"

namespace pcw {

constexpr int MAXL = 14;
constexpr int MAXB = 1 + 3 * MAXL;
constexpr int MAXW = 4;  // mask words: m <= 256

enum : int { ERR_ARENA = 1, ERR_ROWLEN = 2, ERR_INDEX = 4, ERR_QUEUE = 8 };

// ------------------------------------------------------------------------------------------
// Per-operator device view (passed by value).
// ------------------------------------------------------------------------------------------
template <typename T>
struct OpDev {
    int d, n, L, Lf, r, m, gap, order, nb;
    int64_t N;
    const T* u;      // m x Ku kernels
    const T* v;      // m x N windows
    const T* taps;   // h[0..Lf), then g at positions 2-Lf..1 stored as [Lf..2Lf)
    const T* wav;    // base wavelets (unwrapped): level j at wofs[j]: phi [len_j], psi [len_j]
    int wofs[MAXL + 2];
    const T* F;      // filtered base wavelets: band b at Foff[b], layout [k][R0][R1]
    int64_t Foff[MAXB];
    const int64_t* row_ptr;
    T* theta;
    __nv_bfloat16* theta16;
    const unsigned long long* masks;  // [tile][mwords]
    int mwords, ts0, ts1, tpa0, tpa1;
    int* err;
    const void* wl;  // per-pixel window list: slot s of pixel x at wl[s * N + x] (WSlot<T>)
    int wl_slots;    // slots per pixel (the most nonzero windows at any pixel)
    T* sf;           // 2-D: stage-1 values s of every row (band b at Soff[b], row rl at + rl * RR), or null
    int64_t Soff[MAXB];
};

// One nonzero window at a pixel: term index and value (8 bytes for FP32, 16 for FP64).
template <typename T>
struct WSlot;
template <>
struct __align__(8) WSlot<float> {
    int k;
    float v;
};
template <>
struct __align__(16) WSlot<double> {
    long long k;
    double v;
};

__device__ __forceinline__ WSlot<float> load_slot(const WSlot<float>* p)
{
    const int2 r = __ldg(reinterpret_cast<const int2*>(p));
    WSlot<float> w;
    w.k = r.x;
    w.v = __int_as_float(r.y);
    return w;
}
__device__ __forceinline__ WSlot<double> load_slot(const WSlot<double>* p)
{
    const longlong2 r = __ldg(reinterpret_cast<const longlong2*>(p));
    WSlot<double> w;
    w.k = r.x;
    w.v = __longlong_as_double(r.y);
    return w;
}

// Slots needed: the largest number of nonzero windows at one pixel (atomicMax into *out).
template <typename T>
__global__ void k_window_count(const T* __restrict__ v, int m, int64_t N, int* __restrict__ out)
{
    const int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int c = 0;
    if (x < N)
        for (int k = 0; k < m; ++k) c += (v[(int64_t)k * N + x] != T(0));
    c = __reduce_max_sync(0xffffffffu, (unsigned)c);
    if ((threadIdx.x & 31) == 0) atomicMax(out, c);
}

// Per-pixel list of the nonzero windows in increasing k; unused slots hold (0, 0).
template <typename T>
__global__ void k_window_list(const T* __restrict__ v, int m, int64_t N, int slots, WSlot<T>* __restrict__ wl)
{
    const int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (x >= N) return;
    int c = 0;
    for (int k = 0; k < m; ++k) {
        const T val = v[(int64_t)k * N + x];
        if (val != T(0) && c < slots) {
            WSlot<T> w;
            w.k = k;
            w.v = val;
            wl[(int64_t)c * N + x] = w;
            ++c;
        }
    }
    for (; c < slots; ++c) {
        WSlot<T> w;
        w.k = 0;
        w.v = T(0);
        wl[(int64_t)c * N + x] = w;
    }
}

// Per-band launch parameters of k_assemble (one launch per row band, or one queue item).
struct AsmCfg {
    int b;       // band of the stored rows
    int row0;    // first row (within band) of this launch
    int rows;    // rows in this launch
    int gt;      // threads per row group (32, 64, 128, 256)
    int rpc;     // row groups per CTA
    int batch;   // pixel rows of s per stage-1 step (2-D)
    int arena;   // elements of T per row group
    int filt;    // elements of T of the filter area (2 Lf + len of the stage-1 scaling filter)
};

template <typename T>
struct KahanAcc {  // FP64: plain sum
    T s;
    __device__ __forceinline__ void init() { s = T(0); }
    __device__ __forceinline__ void add(T x) { s += x; }
    __device__ __forceinline__ T get() const { return s; }
};
template <>
struct KahanAcc<float> {  // compensated summation (Kahan 1965)
    float s, c;
    __device__ __forceinline__ void init()
    {
        s = 0.f;
        c = 0.f;
    }
    __device__ __forceinline__ void add(float x)
    {
        float y = __fsub_rn(x, c);
        float t = __fadd_rn(s, y);
        c = __fsub_rn(__fsub_rn(t, s), y);
        s = t;
    }
    __device__ __forceinline__ float get() const { return s; }
};

__device__ __forceinline__ void group_sync(int gt, int gid)
{
    if (gt <= 32)
        __syncwarp();
    else
        asm volatile("bar.sync %0, %1;" ::"r"(gid + 1), "r"(gt) : "memory");
}

__device__ __forceinline__ void flag_error(int* err, int bits)
{
    if (err) atomicOr(err, bits);
}

// ------------------------------------------------------------------------------------------
// Base wavelets by the FP64 cascade (Section 2.1):
//   phi_{1,0} = h,  psi_{1,0}(x) = g(x);
//   phi_{j,0}(x) = sum_n h[n] phi_{j-1,0}(x - 2^(j-1) n),  psi_{j,0}(x) = sum_n g[n] phi_{j-1,0}(x - 2^(j-1) n)
// stored unwrapped: phi_j[i] at x = i, psi_j[i] at x = off(j,1) + i.  One CTA.
// ------------------------------------------------------------------------------------------
__global__ void k_base_wavelets(const double* __restrict__ h, int Lf, int L, double* __restrict__ wav)
{
    int base_prev = 0, base = 0;
    for (int j = 1; j <= L; ++j) {
        const int len = wav_len(j, Lf);
        if (j == 1) {
            for (int i = threadIdx.x; i < len; i += blockDim.x) {
                wav[base + i] = h[i];
                const int x = (2 - Lf) + i;  // g(x) = (-1)^(1-x) h[1-x]
                const double s = ((1 - x) & 1) ? -1.0 : 1.0;
                wav[base + len + i] = s * h[1 - x];
            }
        } else {
            const int lenp = wav_len(j - 1, Lf), step = 1 << (j - 1), offp = wav_off(j, 1, Lf);
            const double* phip = wav + base_prev;
            for (int i = threadIdx.x; i < len; i += blockDim.x) {
                double sp = 0.0, sq = 0.0;
                for (int q = 0; q < Lf; ++q) {  // low-pass tap n = q
                    const int y = i - step * q;
                    if (y >= 0 && y < lenp) sp += h[q] * phip[y];
                }
                for (int q = 2 - Lf; q <= 1; ++q) {  // high-pass tap n = q
                    const int y = offp + i - step * q;
                    const double s = ((1 - q) & 1) ? -1.0 : 1.0;
                    if (y >= 0 && y < lenp) sq += s * h[1 - q] * phip[y];
                }
                wav[base + i] = sp;
                wav[base + len + i] = sq;
            }
        }
        __syncthreads();
        base_prev = base;
        base += 2 * len;
    }
}

template <typename T>
__global__ void k_cast(const double* __restrict__ in, T* __restrict__ out, int64_t count)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (T)in[i];
}

// taps in T: h then g (g[2-Lf+i] at index Lf+i)
template <typename T>
__global__ void k_taps(const double* __restrict__ h, int Lf, T* __restrict__ out)
{
    int i = threadIdx.x;
    if (i < Lf) {
        out[i] = (T)h[i];
        const int x = (2 - Lf) + i;
        const double s = ((1 - x) & 1) ? -1.0 : 1.0;
        out[Lf + i] = (T)(s * h[1 - x]);
    }
}

// ------------------------------------------------------------------------------------------
// Filtered base wavelets.  For band b (level j, factors e0, e1) and term k the region is
// supp rho widened by r: unfolded extents U = len_j + 2r per axis, local coordinate q <-> pixel
// x = off(j,e) - r + q.  kappa_k(t) = u_k(-t) in the paper's order (adjoint of the
// convolution), u_k(t) otherwise.
//   pass 1: G[t0][q1] = sum_{t1} kappa_k(t0, t1) rho^{e1}_j(q1 - r - t1)
//   pass 2: F[p0][p1] = sum_{q0 = p0 mod n} sum_{q1 = p1 mod n} sum_{t0} G[t0][q1] rho^{e0}_j(q0 - r - t0)
// (fold mod n when U >= n: the periodised wavelet).  1-D: t0 = 0 and F[p1] = sum G[0][q1].
// ------------------------------------------------------------------------------------------
struct FiltBand {
    int j, e0, e1, U0, U1, R0, R1;
    int64_t Goff, Foff;
};
struct FiltDev {
    int nb, d, n, r, m, Lf, order;
    int wofs[MAXL + 2];
    FiltBand band[MAXB];
};

template <typename T>
__global__ void k_filtered_pass1(const __grid_constant__ FiltDev fd, const T* __restrict__ u,
                                 const T* __restrict__ wav, T* __restrict__ G, int staged)
{
    extern __shared__ __align__(16) unsigned char fsm_raw[];
    const int bk = blockIdx.y;
    const int b = bk / fd.m, k = bk % fd.m;
    const FiltBand& B = fd.band[b];
    const int K = 2 * fd.r + 1, K0 = (fd.d == 2) ? K : 1;
    const int tot = K0 * B.U1;
    const int len = wav_len(B.j, fd.Lf);
    const T* rho1 = wav + fd.wofs[B.j] + (B.e1 ? len : 0);
    const int Ku = (fd.d == 2) ? K * K : K;
    const T* uk = u + (int64_t)k * Ku;
    if ((int)(blockIdx.x * blockDim.x) >= tot) return;  // a block with no outputs (smaller bands)
    if (staged) {
        // the block's kernel stencil and 1-D factor, staged once in shared memory
        T* su = reinterpret_cast<T*>(fsm_raw);
        T* sr = su + Ku;
        for (int i = threadIdx.x; i < Ku + len; i += blockDim.x) {
            if (i < Ku)
                su[i] = uk[i];
            else
                sr[i - Ku] = rho1[i - Ku];
        }
        __syncthreads();
        uk = su;
        rho1 = sr;
    }
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= tot) return;
    const int t0i = idx / B.U1, q1 = idx % B.U1;
    KahanAcc<T> acc;
    acc.init();
    const int t0 = t0i - fd.r;
    for (int t1 = -fd.r; t1 <= fd.r; ++t1) {
        const int y = q1 - fd.r - t1;
        if (y < 0 || y >= len) continue;
        const int tt0 = fd.order == 0 ? -t0 : t0, tt1 = fd.order == 0 ? -t1 : t1;
        const int ui = (fd.d == 2) ? (tt0 + fd.r) * K + (tt1 + fd.r) : (tt1 + fd.r);
        acc.add(uk[ui] * rho1[y]);
    }
    G[B.Goff + ((int64_t)k * K0 + t0i) * B.U1 + q1] = acc.get();
}

template <typename T>
__global__ void k_filtered_pass2(const __grid_constant__ FiltDev fd, const T* __restrict__ wav,
                                 const T* __restrict__ G, T* __restrict__ F, int staged)
{
    extern __shared__ __align__(16) unsigned char fsm_raw[];
    const int bk = blockIdx.y;
    const int b = bk / fd.m, k = bk % fd.m;
    const FiltBand& B = fd.band[b];
    const int tot = B.R0 * B.R1;
    const int K = 2 * fd.r + 1, K0 = (fd.d == 2) ? K : 1;
    const int len = wav_len(B.j, fd.Lf);
    const T* rho0 = wav + fd.wofs[B.j] + (B.e0 ? len : 0);
    const T* Gk = G + B.Goff + (int64_t)k * K0 * B.U1;
    if ((int)(blockIdx.x * blockDim.x) >= tot) return;  // a block with no outputs (smaller bands)
    if (staged) {
        // the band's 1-D factor, staged in shared memory (the pass-1 results are read along the
        // row, coalesced, by consecutive threads)
        T* sr = reinterpret_cast<T*>(fsm_raw);
        for (int i = threadIdx.x; i < len; i += blockDim.x) sr[i] = rho0[i];
        __syncthreads();
        rho0 = sr;
    }
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= tot) return;
    const int p0 = idx / B.R1, p1 = idx % B.R1;
    KahanAcc<T> acc;
    acc.init();
    for (int q1 = p1; q1 < B.U1; q1 += fd.n) {
        if (fd.d == 1) {
            acc.add(Gk[q1]);
        } else {
            for (int q0 = p0; q0 < B.U0; q0 += fd.n) {
                for (int t0i = 0; t0i < K; ++t0i) {
                    const int y = q0 - fd.r - (t0i - fd.r);
                    if (y < 0 || y >= len) continue;
                    acc.add(Gk[(int64_t)t0i * B.U1 + q1] * rho0[y]);
                }
            }
        }
    }
    F[B.Foff + (int64_t)k * tot + idx] = acc.get();
}

// ------------------------------------------------------------------------------------------
// Tile masks: bit k of mask[tile] is set when v_k is nonzero somewhere on the tile.
// One CTA per tile, one pixel per thread (ts0 * ts1 <= blockDim).
// ------------------------------------------------------------------------------------------
template <typename T>
__global__ void k_tile_masks(const T* __restrict__ v, int d, int n, int m, int ts0, int ts1, int tpa1,
                             int mwords, unsigned long long* __restrict__ masks)
{
    const int tile = blockIdx.x;
    const int tr = tile / tpa1, tc = tile % tpa1;
    const int i = threadIdx.x;
    const int p0 = tr * ts0 + i / ts1, p1 = tc * ts1 + i % ts1;
    const bool inside = i < ts0 * ts1;
    const int64_t pix = (d == 2) ? (int64_t)p0 * n + p1 : p1;
    const int64_t N = (d == 2) ? (int64_t)n * n : n;
    for (int w = 0; w < mwords; ++w) {
        unsigned long long word = 0;
        for (int kk = 0; kk < 64 && w * 64 + kk < m; ++kk) {
            const int k = w * 64 + kk;
            const int nz = inside && v[(int64_t)k * N + pix] != T(0);
            if (__syncthreads_or(nz)) word |= 1ull << kk;
        }
        if (threadIdx.x == 0) masks[(int64_t)tile * mwords + w] = word;
    }
}

// ------------------------------------------------------------------------------------------
// Stride-S filter on one axis of a group-shared array (Range conventions of pcw_geom.cuh):
//   out[c] = sum_{i<len} f[i] * in[S*(ro.lo + c) + off + i]   (in indexed from ri.lo)
// Non-full output: inputs outside [ri.lo, ri.lo + ri.cnt) are zero.  Full output: periodic.
// ------------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T filt(const T* in, int istride, Range ri, int n_in, Range ro, int c,
                                  const T* f, int len, int S, int off)
{
    const int x0 = S * (ro.lo + c) + off - ri.lo;
    T acc = T(0);
    if (!ro.full) {
        const int ilo = x0 < 0 ? -x0 : 0;
        const int ihi = min(len, ri.cnt - x0);
        for (int i = ilo; i < ihi; ++i) acc = fma(f[i], in[(x0 + i) * istride], acc);
    } else {
        for (int i = 0; i < len; ++i) {
            const int p = pmod(x0 + i, n_in);
            if (p < ri.cnt) acc = fma(f[i], in[p * istride], acc);
        }
    }
    return acc;
}

// Writes the stencil block of column band b2 (level jj, factors e0, e1) from a band array of
// shape r0.cnt x r1.cnt to the row's storage.
template <typename T, int DIM>
__device__ __forceinline__ void write_block(const OpDev<T>& op, const T* Zb, Range r0, Range r1, int jj, int e0,
                                            int e1, int64_t dst, int j, int eo0, int eo1, int l0, int l1,
                                            int tid, int gt)
{
    const int dense = op.gap < 0;
    int f0 = 0, W0 = 1, f1, W1;
    stencil(j, eo1, l1, jj, e1, op.r, op.Lf, op.n, dense, &f1, &W1);
    if (DIM == 2) stencil(j, eo0, l0, jj, e0, op.r, op.Lf, op.n, dense, &f0, &W0);
    const int nj = op.n >> jj;
    const int tot = W0 * W1;
    for (int idx = tid; idx < tot; idx += gt) {
        const int a = idx / W1, bb = idx - a * W1;
        const int p1 = pmod(f1 + bb - r1.lo, nj);
        bool ok = r1.full || p1 < r1.cnt;
        int p0 = 0;
        if (DIM == 2) {
            p0 = pmod(f0 + a - r0.lo, nj);
            ok = ok && (r0.full || p0 < r0.cnt);
        }
        const T val = ok ? Zb[p0 * r1.cnt + p1] : T(0);
        op.theta[dst + idx] = val;
        if (op.theta16) op.theta16[dst + idx] = __float2bfloat16_rn((float)val);
    }
}

// ------------------------------------------------------------------------------------------
// 1-D assembly: fused window-multiply + localized forward transform, one stored row per thread
// group.  hS, gS: taps in shared memory; boff: the group's block-offset table (nb + 1 ints);
// arena: the group's cfg.arena elements.
// ------------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void asm1d_row(const OpDev<T>& op, const AsmCfg& cfg, int rl, const T* hS, const T* gS,
                                          int* boff, T* arena, int gid, int tid)
{
    const int gt = cfg.gt;
    const int n = op.n, L = op.L, Lf = op.Lf, r = op.r;
    const int dense = op.gap < 0;
    const Band Bo = band_info(1, n, L, cfg.b);
    const int j = Bo.j;
    const int jlo = dense ? 1 : max(1, j - op.gap);
    const int jhi = dense ? L : min(L, j + op.gap);
    T* const arena_end = arena + cfg.arena;
    const int l1 = rl;
    const Range A1 = region0(j, Bo.e1, l1, r, Lf, n);
    const int g1 = pmod(A1.lo, n);
    const int64_t srow = Bo.off + rl;
    const int64_t row_base = op.row_ptr[srow];
    if (tid == 0) {
        int acc = 0;
        for (int b2 = 0; b2 < op.nb; ++b2) {
            boff[b2] = acc;
            if (block_kept(1, n, L, op.gap, cfg.b, b2)) acc += (int)block_count(1, n, L, Lf, r, op.gap, cfg.b, 0, l1, b2);
        }
        boff[op.nb] = acc;
        if ((int64_t)acc != op.row_ptr[srow + 1] - row_base) flag_error(op.err, ERR_ROWLEN);
    }
    // windows nonzero on the region: OR of the tile masks it covers (every warp reduces alone)
    unsigned long long mw[MAXW];
#pragma unroll
    for (int w = 0; w < MAXW; ++w) mw[w] = 0ull;
    {
        const int lane = threadIdx.x & 31;
        const int ts1 = op.ts1;
        const int s1 = g1 / ts1;
        const int nt1 = min(op.tpa1, (g1 % ts1 + A1.cnt + ts1 - 1) / ts1);
        for (int i = lane; i < nt1; i += 32) {
            const int t1 = (s1 + i) % op.tpa1;
            const unsigned long long* mp = op.masks + (int64_t)t1 * op.mwords;
#pragma unroll
            for (int w = 0; w < MAXW; ++w)
                if (w < op.mwords) mw[w] |= mp[w];
        }
#pragma unroll
        for (int w = 0; w < MAXW; ++w) {
            const unsigned lo = __reduce_or_sync(0xffffffffu, (unsigned)mw[w]);
            const unsigned hi = __reduce_or_sync(0xffffffffu, (unsigned)(mw[w] >> 32));
            mw[w] = ((unsigned long long)hi << 32) | lo;
        }
    }
    const T* Fb = op.F + op.Foff[cfg.b];
    const int RR = A1.cnt;
    T* X = arena;
    if (A1.cnt > cfg.arena) {
        flag_error(op.err, ERR_ARENA);
        return;
    }
    // s(q) = sum_k v_k(g + q) F_{k,b}(q), compensated over k
    for (int q1 = tid; q1 < A1.cnt; q1 += gt) {
        const int gx = (g1 + q1) & (n - 1);
        KahanAcc<T> acc;
        acc.init();
#pragma unroll
        for (int w = 0; w < MAXW; ++w) {
            unsigned long long bits = mw[w];
            while (bits) {
                const int k = w * 64 + __ffsll((long long)bits) - 1;
                bits &= bits - 1;
                const T vk = __ldg(op.v + (int64_t)k * op.N + gx);
                if (vk != T(0)) acc.add(vk * __ldg(Fb + (int64_t)k * RR + q1));
            }
        }
        X[q1] = acc.get();
    }
    group_sync(gt, gid);
    if ((int64_t)boff[op.nb] != op.row_ptr[srow + 1] - row_base) return;  // flagged above
    // cascade with (a|d) outputs alternating between the arena ends
    Range cur = A1;
    const T* in = X;
    int n_in = n;
    bool out_top = true;
    int prev_out = A1.cnt;
    for (int jj = 1; jj <= jhi; ++jj) {
        const Range nx = range_cascade(cur, Lf, n >> jj);
        if (2 * nx.cnt + prev_out > (int)(arena_end - arena)) {
            flag_error(op.err, ERR_ARENA);
            return;
        }
        T* out = out_top ? (arena_end - 2 * nx.cnt) : arena;
        for (int c = tid; c < nx.cnt; c += gt) {
            out[c] = filt(in, 1, cur, n_in, nx, c, hS, Lf, 2, 0);
            out[nx.cnt + c] = filt(in, 1, cur, n_in, nx, c, gS, Lf, 2, 2 - Lf);
        }
        group_sync(gt, gid);
        if (jj >= jlo) {
            const int b2 = band_of_level(1, L, jj, 0);
            write_block<T, 1>(op, out + nx.cnt, Range{0, 1, 0}, nx, jj, 0, 1, row_base + boff[b2], j, 0, Bo.e1, 0, l1,
                              tid, gt);
            if (jj == L)
                write_block<T, 1>(op, out, Range{0, 1, 0}, nx, jj, 0, 0, row_base + boff[0], j, 0, Bo.e1, 0, l1, tid,
                                  gt);
        }
        in = out;
        cur = nx;
        n_in = n >> jj;
        out_top = !out_top;
        prev_out = 2 * nx.cnt;
    }
}

// Shared-memory layout of the row kernels: filters (cfg.filt elements of T) | per group a meta
// area of META_INTS ints | per group an arena of cfg.arena elements of T.
// meta area of a 2-D row group: block offsets [MAXB + 1], the stencil window of every kept
// column band (f0, W0, f1, W1) [4 MAXB], active terms (bytes) [64 ints], their count
constexpr int WIN_OFF = MAXB + 1;
constexpr int ACT_OFF = WIN_OFF + 4 * MAXB;
constexpr int NACT_OFF = ACT_OFF + 64;
constexpr int META_INTS = (NACT_OFF + 1 + 3) / 4 * 4;
static_assert(NACT_OFF < META_INTS, "meta layout");

template <typename T>
__global__ void __launch_bounds__(256) k_assemble1d(const __grid_constant__ OpDev<T> op, const AsmCfg cfg)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int gt = cfg.gt;
    const int gid = threadIdx.x / gt, tid = threadIdx.x % gt;
    T* fS = reinterpret_cast<T*>(smem_raw);
    int* meta = reinterpret_cast<int*>(smem_raw + sizeof(T) * cfg.filt) + gid * META_INTS;
    T* arena = reinterpret_cast<T*>(smem_raw + sizeof(T) * cfg.filt + sizeof(int) * cfg.rpc * META_INTS) +
               (int64_t)gid * cfg.arena;
    for (int i = threadIdx.x; i < 2 * op.Lf; i += blockDim.x) fS[i] = op.taps[i];
    __syncthreads();
    const int rloc = blockIdx.x * cfg.rpc + gid;
    if (rloc >= cfg.rows) return;
    asm1d_row<T>(op, cfg, cfg.row0 + rloc, fS, fS + op.Lf, meta, arena, gid, tid);
}

// ------------------------------------------------------------------------------------------
// Adjoint (backward).  The transpose of filt(): for an input position p,
//   in_bar[p] = sum over (c, i) with S*(ro.lo + c) + off + i = ri.lo + p (mod n_in when the
//   output is full) of f[i] * out_bar[c].
// ------------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T filt_adj(const T* outb, int ostride, Range ri, Range ro, int n_out, int p, const T* f,
                                      int len, int S, int off)
{
    const int x = ri.lo + p - off;  // = S*y + i
    T acc = T(0);
    for (int i = pmod(x, S); i < len; i += S) {
        const int y = (x - i) / S;  // exact
        int c = y - ro.lo;
        if (!ro.full) {
            if ((unsigned)c >= (unsigned)ro.cnt) continue;
        } else {
            c = pmod(c, n_out);
        }
        acc = fma(f[i], outb[c * ostride], acc);
    }
    return acc;
}

// Scatters the row's dL/dTheta entries of column band b2 into a zeroed band array (transpose
// of write_block).
template <typename T, int DIM>
__device__ __forceinline__ void read_block(const OpDev<T>& op, const T* __restrict__ Gr, T* Zb, Range r0, Range r1,
                                           int jj, int e0, int e1, int64_t src, int j, int eo0, int eo1, int l0,
                                           int l1, int tid, int gt)
{
    const int dense = op.gap < 0;
    int f0 = 0, W0 = 1, f1, W1;
    stencil(j, eo1, l1, jj, e1, op.r, op.Lf, op.n, dense, &f1, &W1);
    if (DIM == 2) stencil(j, eo0, l0, jj, e0, op.r, op.Lf, op.n, dense, &f0, &W0);
    const int nj = op.n >> jj;
    const int tot = W0 * W1;
    for (int idx = tid; idx < tot; idx += gt) {
        const int a = idx / W1, bb = idx - a * W1;
        const int p1 = pmod(f1 + bb - r1.lo, nj);
        bool ok = r1.full || p1 < r1.cnt;
        int p0 = 0;
        if (DIM == 2) {
            p0 = pmod(f0 + a - r0.lo, nj);
            ok = ok && (r0.full || p0 < r0.cnt);
        }
        if (ok) Zb[p0 * r1.cnt + p1] = Gr[src + idx];
    }
}

// One stored row per thread group: dL/ds on the row's region by the transposed localized
// transform of the row's dL/dTheta, then
//   dL/dv_k(x) += F_{k,b}(x - shift) dL/ds(x)   (every k)
//   dL/dF_{k,b}(q) += v_k(q + shift) dL/ds(q)   (k with v_k nonzero on the region)
// with atomics into dv (m x N) and dF (layout of F).
template <typename T, int DIM>
__global__ void __launch_bounds__(256) k_backward(const __grid_constant__ OpDev<T> op, const AsmCfg cfg,
                                                  const T* __restrict__ Gth, T* __restrict__ dv, T* __restrict__ dF)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int gt = cfg.gt;
    const int gid = threadIdx.x / gt, tid = threadIdx.x % gt;
    const int n = op.n, L = op.L, Lf = op.Lf, r = op.r;
    const int dense = op.gap < 0;
    const Band Bo = band_info(DIM, n, L, cfg.b);
    const int j = Bo.j;
    const int jlo = dense ? 1 : max(1, j - op.gap);
    const int jhi = dense ? L : min(L, j + op.gap);
    const int k0 = (DIM == 2) ? jlo - 1 : 0;

    T* fS = reinterpret_cast<T*>(smem_raw);
    T* hS = fS;
    T* gS = fS + Lf;
    T* phiS = fS + 2 * Lf;
    const int lenk = (k0 > 0) ? wav_len(k0, Lf) : 0;
    int* boffAll = reinterpret_cast<int*>(smem_raw + sizeof(T) * cfg.filt);
    int* boff = boffAll + gid * (MAXB + 1);
    T* arena = reinterpret_cast<T*>(smem_raw + sizeof(T) * cfg.filt + sizeof(int) * cfg.rpc * (MAXB + 1));
    arena += (int64_t)gid * cfg.arena;
    T* const arena_end = arena + cfg.arena;
    const int A = cfg.arena;

    for (int i = threadIdx.x; i < 2 * Lf; i += blockDim.x) fS[i] = op.taps[i];
    for (int i = threadIdx.x; i < lenk; i += blockDim.x) phiS[i] = op.wav[op.wofs[k0] + i];
    __syncthreads();

    const int rl = cfg.row0 + blockIdx.x * cfg.rpc + gid;
    if (blockIdx.x * cfg.rpc + gid >= cfg.rows) return;
    const int l0 = (DIM == 2) ? rl / Bo.nj : 0;
    const int l1 = (DIM == 2) ? rl % Bo.nj : rl;
    const Range A1 = region0(j, Bo.e1, l1, r, Lf, n);
    const Range A0 = (DIM == 2) ? region0(j, Bo.e0, l0, r, Lf, n) : Range{0, 1, 0};
    const int g0 = (DIM == 2) ? pmod(A0.lo, n) : 0;
    const int g1 = pmod(A1.lo, n);
    const int64_t srow = Bo.off + rl;
    const int64_t row_base = op.row_ptr[srow];
    if (tid == 0) {
        int acc = 0;
        for (int b2 = 0; b2 < op.nb; ++b2) {
            boff[b2] = acc;
            if (block_kept(DIM, n, L, op.gap, cfg.b, b2))
                acc += (int)block_count(DIM, n, L, Lf, r, op.gap, cfg.b, l0, l1, b2);
        }
        boff[op.nb] = acc;
        if ((int64_t)acc != op.row_ptr[srow + 1] - row_base) flag_error(op.err, ERR_ROWLEN);
    }
    unsigned long long mw[MAXW];
#pragma unroll
    for (int w = 0; w < MAXW; ++w) mw[w] = 0ull;
    {
        const int lane = threadIdx.x & 31;
        const int ts0 = op.ts0, ts1 = op.ts1;
        const int s0 = g0 / ts0, s1 = g1 / ts1;
        const int nt0 = (DIM == 2) ? min(op.tpa0, (g0 % ts0 + A0.cnt + ts0 - 1) / ts0) : 1;
        const int nt1 = min(op.tpa1, (g1 % ts1 + A1.cnt + ts1 - 1) / ts1);
        for (int i = lane; i < nt0 * nt1; i += 32) {
            const int t0 = (s0 + i / nt1) % op.tpa0, t1 = (s1 + i % nt1) % op.tpa1;
            const unsigned long long* mp = op.masks + ((int64_t)t0 * op.tpa1 + t1) * op.mwords;
#pragma unroll
            for (int w = 0; w < MAXW; ++w)
                if (w < op.mwords) mw[w] |= mp[w];
        }
#pragma unroll
        for (int w = 0; w < MAXW; ++w) {
            const unsigned lo = __reduce_or_sync(0xffffffffu, (unsigned)mw[w]);
            const unsigned hi = __reduce_or_sync(0xffffffffu, (unsigned)(mw[w] >> 32));
            mw[w] = ((unsigned long long)hi << 32) | lo;
        }
    }
    group_sync(gt, gid);
    if ((int64_t)boff[op.nb] != op.row_ptr[srow + 1] - row_base) return;
    const int64_t N = op.N;
    const int64_t Fo = op.Foff[cfg.b];
    const int RR = A0.cnt * A1.cnt;

    // dL/ds(q) -> dv, dF
    auto scatter = [&](int q0, int q1, T sb) {
        int gy = g0 + q0;
        if (gy >= n) gy -= n;
        int gx = g1 + q1;
        if (gx >= n) gx -= n;
        const int64_t pix = (DIM == 2) ? (int64_t)gy * n + gx : gx;
        const int q = q0 * A1.cnt + q1;
        if (sb == T(0)) return;
        for (int k = 0; k < op.m; ++k) {
            const int64_t fi = Fo + (int64_t)k * RR + q;
            atomicAdd(dv + (int64_t)k * N + pix, __ldg(op.F + fi) * sb);
            if ((mw[k >> 6] >> (k & 63)) & 1ull) {
                const T vk = __ldg(op.v + (int64_t)k * N + pix);
                if (vk != T(0)) atomicAdd(dF + fi, vk * sb);
            }
        }
    };

    if (DIM == 1) {
        // ranges of the forward cascade: R(0) = A1, R(jj) = cascade of R(jj-1)
        // level jj's [a|d] sits at the top for odd jj, at the bottom for even jj (forward layout)
        Range Rj = A1;
        Range Rs[MAXL + 2];
        Rs[0] = A1;
        for (int jj = 1; jj <= jhi; ++jj) {
            Rj = range_cascade(Rj, Lf, n >> jj);
            Rs[jj] = Rj;
        }
        for (int jj = jhi; jj >= 1; --jj) {
            const Range R = Rs[jj], P = Rs[jj - 1];
            if (2 * R.cnt + ((jj == 1) ? P.cnt : 2 * P.cnt) > A) {
                flag_error(op.err, ERR_ARENA);
                return;
            }
            T* buf = (jj & 1) ? (arena_end - 2 * R.cnt) : arena;
            T* prev = (jj & 1) ? arena : (arena_end - 2 * P.cnt);  // level jj-1 (a part first), or X
            for (int c = tid; c < R.cnt; c += gt) {
                if (jj == jhi) buf[c] = T(0);
                buf[R.cnt + c] = T(0);
            }
            group_sync(gt, gid);
            if (jj >= jlo) read_block<T, 1>(op, Gth, buf + R.cnt, Range{0, 1, 0}, R, jj, 0, 1,
                                           row_base + boff[band_of_level(1, L, jj, 0)], j, 0, Bo.e1, 0, l1, tid, gt);
            if (jj == jhi && jj == L)
                read_block<T, 1>(op, Gth, buf, Range{0, 1, 0}, R, jj, 0, 0, row_base + boff[0], j, 0, Bo.e1, 0, l1,
                                 tid, gt);
            group_sync(gt, gid);
            for (int p = tid; p < P.cnt; p += gt)
                prev[p] = filt_adj(buf, 1, P, R, n >> jj, p, hS, Lf, 2, 0) +
                          filt_adj(buf + R.cnt, 1, P, R, n >> jj, p, gS, Lf, 2, 2 - Lf);
            group_sync(gt, gid);
        }
        for (int q1 = tid; q1 < A1.cnt; q1 += gt) scatter(0, q1, arena[q1]);
        return;
    }

    // ---------------- 2-D ----------------
    Range c0, c1;
    int S1, n1;
    if (k0 == 0) {
        n1 = n >> 1;
        S1 = 2;
        c0 = range_cascade(A0, Lf, n1);
        c1 = range_cascade(A1, Lf, n1);
    } else {
        n1 = n >> k0;
        S1 = 1 << k0;
        c0 = range_filter(A0, S1, 0, lenk, n1);
        c1 = range_filter(A1, S1, 0, lenk, n1);
    }
    const int lvl0 = (k0 == 0) ? 1 : k0;
    Range Q0[MAXL + 2], Q1[MAXL + 2];
    Q0[lvl0] = c0;
    Q1[lvl0] = c1;
    for (int jj = lvl0 + 1; jj <= jhi; ++jj) {
        Q0[jj] = range_cascade(Q0[jj - 1], Lf, n >> jj);
        Q1[jj] = range_cascade(Q1[jj - 1], Lf, n >> jj);
    }
    T* Z = arena;
    // cascade levels, coarse to fine
    for (int jj = jhi; jj >= lvl0 + 1; --jj) {
        const int nj = n >> jj;
        const Range q0r = Q0[jj], q1r = Q1[jj], p0 = Q0[jj - 1], p1 = Q1[jj - 1];
        const int zq = q0r.cnt * q1r.cnt, ysz = 2 * p0.cnt * q1r.cnt;
        if (4 * zq + ysz > A || p0.cnt * p1.cnt + ysz > A) {
            flag_error(op.err, ERR_ARENA);
            return;
        }
        for (int e = tid; e < ((jj == jhi) ? 4 : 3) * zq; e += gt) Z[((jj == jhi) ? 0 : zq) + e] = T(0);
        group_sync(gt, gid);
        for (int t = 0; t < 3; ++t)
            read_block<T, 2>(op, Gth, Z + (1 + t) * zq, q0r, q1r, jj, t >= 1 ? 1 : 0, t == 1 ? 0 : 1,
                             row_base + boff[band_of_level(2, L, jj, t)], j, Bo.e0, Bo.e1, l0, l1, tid, gt);
        if (jj == jhi && jj == L)
            read_block<T, 2>(op, Gth, Z, q0r, q1r, jj, 0, 0, row_base + boff[0], j, Bo.e0, Bo.e1, l0, l1, tid, gt);
        group_sync(gt, gid);
        T* Yl = arena_end - ysz;
        T* Yh = Yl + p0.cnt * q1r.cnt;
        for (int e = tid; e < p0.cnt * q1r.cnt; e += gt) {
            const int a = e / q1r.cnt, c = e - a * q1r.cnt;
            Yl[e] = filt_adj(Z + c, q1r.cnt, p0, q0r, nj, a, hS, Lf, 2, 0) +
                    filt_adj(Z + 2 * zq + c, q1r.cnt, p0, q0r, nj, a, gS, Lf, 2, 2 - Lf);
            Yh[e] = filt_adj(Z + zq + c, q1r.cnt, p0, q0r, nj, a, hS, Lf, 2, 0) +
                    filt_adj(Z + 3 * zq + c, q1r.cnt, p0, q0r, nj, a, gS, Lf, 2, 2 - Lf);
        }
        group_sync(gt, gid);
        for (int e = tid; e < p0.cnt * p1.cnt; e += gt) {
            const int a = e / p1.cnt, b = e - a * p1.cnt;
            Z[e] = filt_adj(Yl + a * q1r.cnt, 1, p1, q1r, nj, b, hS, Lf, 2, 0) +
                   filt_adj(Yh + a * q1r.cnt, 1, p1, q1r, nj, b, gS, Lf, 2, 2 - Lf);
        }
        group_sync(gt, gid);
    }
    // stage 1 (level 1 with its detail bands, or LL of level k0)
    const int zb = c0.cnt * c1.cnt;
    const int nY = (k0 == 0) ? 2 : 1;
    const int Ysz = nY * A0.cnt * c1.cnt;
    if (((k0 == 0) ? 4 : 1) * zb + Ysz > A) {
        flag_error(op.err, ERR_ARENA);
        return;
    }
    if (k0 == 0) {
        const bool top = (jhi == 1);
        for (int e = tid; e < (top ? 4 : 3) * zb; e += gt) Z[(top ? 0 : zb) + e] = T(0);
        group_sync(gt, gid);
        for (int t = 0; t < 3; ++t)
            read_block<T, 2>(op, Gth, Z + (1 + t) * zb, c0, c1, 1, t >= 1 ? 1 : 0, t == 1 ? 0 : 1,
                             row_base + boff[band_of_level(2, L, 1, t)], j, Bo.e0, Bo.e1, l0, l1, tid, gt);
        if (L == 1) read_block<T, 2>(op, Gth, Z, c0, c1, 1, 0, 0, row_base + boff[0], j, Bo.e0, Bo.e1, l0, l1, tid, gt);
        group_sync(gt, gid);
    }
    T* YL = arena_end - Ysz;
    T* YH = YL + A0.cnt * c1.cnt;
    for (int e = tid; e < A0.cnt * c1.cnt; e += gt) {
        const int q0 = e / c1.cnt, c = e - q0 * c1.cnt;
        if (k0 == 0) {
            YL[e] = filt_adj(Z + c, c1.cnt, A0, c0, n1, q0, hS, Lf, 2, 0) +
                    filt_adj(Z + 2 * zb + c, c1.cnt, A0, c0, n1, q0, gS, Lf, 2, 2 - Lf);
            YH[e] = filt_adj(Z + zb + c, c1.cnt, A0, c0, n1, q0, hS, Lf, 2, 0) +
                    filt_adj(Z + 3 * zb + c, c1.cnt, A0, c0, n1, q0, gS, Lf, 2, 2 - Lf);
        } else {
            YL[e] = filt_adj(Z + c, c1.cnt, A0, c0, n1, q0, phiS, lenk, S1, 0);
        }
    }
    group_sync(gt, gid);
    for (int e = tid; e < RR; e += gt) {
        const int q0 = e / A1.cnt, q1 = e - q0 * A1.cnt;
        T sb;
        if (k0 == 0)
            sb = filt_adj(YL + q0 * c1.cnt, 1, A1, c1, n1, q1, hS, Lf, 2, 0) +
                 filt_adj(YH + q0 * c1.cnt, 1, A1, c1, n1, q1, gS, Lf, 2, 2 - Lf);
        else
            sb = filt_adj(YL + q0 * c1.cnt, 1, A1, c1, n1, q1, phiS, lenk, S1, 0);
        scatter(q0, q1, sb);
    }
}

// Adjoint of the filtered base wavelets.  pass 2^T: dG[t0][q1] = sum_{q0 < U0} dF[q0 mod n][q1 mod n] rho^{e0}_j(q0 - r - t0)
template <typename T>
__global__ void k_dfilt_pass2(const __grid_constant__ FiltDev fd, const T* __restrict__ wav,
                              const T* __restrict__ dF, T* __restrict__ dG)
{
    const int bk = blockIdx.y;
    const int b = bk / fd.m, k = bk % fd.m;
    const FiltBand& B = fd.band[b];
    const int K = 2 * fd.r + 1, K0 = (fd.d == 2) ? K : 1;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= K0 * B.U1) return;
    const int t0i = idx / B.U1, q1 = idx % B.U1;
    const int len = wav_len(B.j, fd.Lf);
    const T* dFk = dF + B.Foff + (int64_t)k * B.R0 * B.R1;
    const int p1 = q1 % fd.n;
    T acc = T(0);
    if (fd.d == 1) {
        acc = dFk[p1];
    } else {
        const T* rho0 = wav + fd.wofs[B.j] + (B.e0 ? len : 0);
        const int qlo = t0i, qhi = min(B.U0, t0i + len);  // rho index q0 - t0i in [0, len)
        for (int q0 = qlo; q0 < qhi; ++q0) acc = fma(dFk[(int64_t)(q0 % fd.n) * B.R1 + p1], rho0[q0 - t0i], acc);
    }
    dG[B.Goff + ((int64_t)k * K0 + t0i) * B.U1 + q1] = acc;
}

// pass 1^T summed over bands: dkappa_k(t0, t1) = sum_b sum_q1 dG_b[t0][q1] rho^{e1}_j(q1 - r - t1);
// du_k(t) = dkappa_k(-t) in the paper's order, dkappa_k(t) otherwise.  One thread per (k, t).
template <typename T>
__global__ void k_dfilt_pass1(const __grid_constant__ FiltDev fd, const T* __restrict__ wav,
                              const T* __restrict__ dG, T* __restrict__ du)
{
    const int K = 2 * fd.r + 1, K0 = (fd.d == 2) ? K : 1, Ku = K0 * K;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= fd.m * Ku) return;
    const int k = idx / Ku, t = idx % Ku;
    const int t0i = t / K, t1i = t % K;
    T acc = T(0);
    for (int b = 0; b < fd.nb; ++b) {
        const FiltBand& B = fd.band[b];
        const int len = wav_len(B.j, fd.Lf);
        const T* rho1 = wav + fd.wofs[B.j] + (B.e1 ? len : 0);
        const T* g = dG + B.Goff + ((int64_t)k * K0 + t0i) * B.U1;
        const int qlo = t1i, qhi = min(B.U1, t1i + len);
        for (int q1 = qlo; q1 < qhi; ++q1) acc = fma(g[q1], rho1[q1 - t1i], acc);
    }
    const int o = (fd.order == 0) ? (Ku - 1 - t) : t;  // flip: index of -t
    du[(int64_t)k * Ku + o] = acc;
}

// ------------------------------------------------------------------------------------------
// y = S x (gather over a stored row) or y = S^T x (scatter with atomics into a zeroed y), S
// the stored matrix: Theta in the paper's order, Theta^T in the convolution-first order, so
// the adjoint apply takes the other direction.  One warp per stored row, NR right-hand
// sides per pass, warp-shuffle reduction of the row sums.  SQ squares the stored values:
// (Theta o Theta)^T 1 = diag(Theta^T Theta).
// ------------------------------------------------------------------------------------------
template <typename TA, typename TV>
__device__ __forceinline__ TA to_acc(TV v) { return (TA)v; }
template <>
__device__ __forceinline__ float to_acc<float, __nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

template <typename TV, typename TA, int NR, bool SQ = false>
__global__ void __launch_bounds__(256) k_apply(const __grid_constant__ OpDev<TA> op, const TV* __restrict__ vals,
                                               const TA* __restrict__ x, int ldx, TA* __restrict__ y, int ldy,
                                               int c0, int nr, int transpose)
{
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int64_t s = warp;
    if (s >= op.N) return;
    const int d = op.d, n = op.n, L = op.L;
    int b = 0;
    Band Bo = band_info(d, n, L, 0);
    for (int bb = op.nb - 1; bb >= 0; --bb) {
        const Band t = band_info(d, n, L, bb);
        const int64_t sz = (d == 2) ? (int64_t)t.nj * t.nj : t.nj;
        if (s >= t.off && s < t.off + sz) {
            b = bb;
            Bo = t;
            break;
        }
    }
    const int rl = (int)(s - Bo.off);
    const int l0 = (d == 2) ? rl / Bo.nj : 0, l1 = (d == 2) ? rl % Bo.nj : rl;
    const int dense = op.gap < 0;
    TA acc[NR];
#pragma unroll
    for (int q = 0; q < NR; ++q) acc[q] = TA(0);
    TA xs[NR];
    if (transpose) {
#pragma unroll
        for (int q = 0; q < NR; ++q) xs[q] = (q < nr) ? x[s * ldx + c0 + q] : TA(0);
    }
    int64_t pos = op.row_ptr[s];
    for (int b2 = 0; b2 < op.nb; ++b2) {
        if (!block_kept(d, n, L, op.gap, b, b2)) continue;
        const Band B2 = band_info(d, n, L, b2);
        int f0 = 0, W0 = 1, f1, W1;
        stencil(Bo.j, Bo.e1, l1, B2.j, B2.e1, op.r, op.Lf, n, dense, &f1, &W1);
        if (d == 2) stencil(Bo.j, Bo.e0, l0, B2.j, B2.e0, op.r, op.Lf, n, dense, &f0, &W0);
        const int nj = B2.nj, tot = W0 * W1;
        for (int idx = lane; idx < tot; idx += 32) {
            const int a = idx / W1, bb = idx - a * W1;
            const int64_t col = B2.off + (int64_t)pmod(f0 + a, nj) * ((d == 2) ? nj : 0) + pmod(f1 + bb, nj);
            TA v = to_acc<TA, TV>(vals[pos + idx]);
            if (SQ) v *= v;
            if (!transpose) {
                const TA* xr = x + col * ldx + c0;
#pragma unroll
                for (int q = 0; q < NR; ++q)
                    if (q < nr) acc[q] = fma(v, xr[q], acc[q]);
            } else {
                TA* yr = y + col * ldy + c0;
#pragma unroll
                for (int q = 0; q < NR; ++q)
                    if (q < nr) atomicAdd(yr + q, v * xs[q]);
            }
        }
        pos += tot;
    }
    if (!transpose) {
#pragma unroll
        for (int q = 0; q < NR; ++q) {
            TA vq = acc[q];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) vq += __shfl_xor_sync(0xffffffffu, vq, o);
            acc[q] = vq;
        }
        if (lane < nr && lane < NR) {
            TA out = acc[0];
#pragma unroll
            for (int q = 1; q < NR; ++q)
                if (lane == q) out = acc[q];
            y[s * ldy + c0 + lane] = out;
        }
    }
}

// Column-block descriptors of every stored row for the one-right-hand-side products: for
// row s, slot k < stride (the most kept blocks of any row band) holds the k-th kept column block (band b2, first translates f0, f1 on
// the torus, extents W0 x W1) packed in 64 bits, 0 after the last one.
//   2-D: W0 [0,14) W1 [14,28) f0 [28,42) f1 [42,56) b2 [56,62)   (n <= 16384, so nj < 2^14)
//   1-D: W1 [0,28) f1 [28,56) b2 [56,62)                          (n <= 2^28)
constexpr int BLK_B2_SHIFT = 56;
template <typename TA>
__global__ void __launch_bounds__(256) k_block_desc(const __grid_constant__ OpDev<TA> op,
                                                    unsigned long long* __restrict__ desc,
                                                    unsigned* __restrict__ boff, int stride)
{
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= op.N) return;
    const int d = op.d, n = op.n, L = op.L;
    int b = 0;
    Band Bo = band_info(d, n, L, 0);
    for (int bb = op.nb - 1; bb >= 0; --bb) {
        const Band t = band_info(d, n, L, bb);
        const int64_t sz = (d == 2) ? (int64_t)t.nj * t.nj : t.nj;
        if (s >= t.off && s < t.off + sz) {
            b = bb;
            Bo = t;
            break;
        }
    }
    const int rl = (int)(s - Bo.off);
    const int l0 = (d == 2) ? rl / Bo.nj : 0, l1 = (d == 2) ? rl % Bo.nj : rl;
    const int dense = op.gap < 0;
    int k = 0;
    unsigned start = 0;
    for (int b2 = 0; b2 < op.nb; ++b2) {
        if (!block_kept(d, n, L, op.gap, b, b2)) continue;
        const Band B2 = band_info(d, n, L, b2);
        int f0 = 0, W0 = 1, f1, W1;
        stencil(Bo.j, Bo.e1, l1, B2.j, B2.e1, op.r, op.Lf, n, dense, &f1, &W1);
        if (d == 2) stencil(Bo.j, Bo.e0, l0, B2.j, B2.e0, op.r, op.Lf, n, dense, &f0, &W0);
        boff[s * stride + k] = start;
        start += (unsigned)(W0 * W1);
        const unsigned long long f0p = (unsigned)pmod(f0, B2.nj), f1p = (unsigned)pmod(f1, B2.nj);
        unsigned long long w;
        if (d == 2)
            w = (unsigned long long)W0 | ((unsigned long long)W1 << 14) | (f0p << 28) | (f1p << 42);
        else
            w = (unsigned long long)W1 | (f1p << 28);
        desc[s * stride + k++] = w | ((unsigned long long)b2 << BLK_B2_SHIFT);
    }
    for (; k < stride; ++k) {
        desc[s * stride + k] = 0ull;
        boff[s * stride + k] = start;
    }
}

// Transposed copy of the stored matrix in the same pattern (the pattern is symmetric):
// valsT[row lambda, column mu] = vals[row mu, column lambda], each row in the stored order, so
// that Theta^T x is a gather with the row pointers and descriptors of Theta.  One warp per
// stored row mu; for its entry (mu, lambda) the block of row lambda that holds band(mu) is slot
// kk of lambda's list (the same for every lambda of one band), and mu's place in it follows from
// that block's first translates.  A place outside the block (a pattern that is not symmetric)
// flags ERR_INDEX and is skipped.
template <typename T>
__global__ void __launch_bounds__(256) k_transpose_theta(const __grid_constant__ OpDev<T> op,
                                                         const unsigned long long* __restrict__ desc,
                                                         const unsigned* __restrict__ boff, int nbands,
                                                         const T* __restrict__ vals, T* __restrict__ valsT)
{
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int64_t s = warp;
    if (s >= op.N) return;
    const int d = op.d, n = op.n, L = op.L;
    int b = 0;
    Band Bo = band_info(d, n, L, 0);
    for (int bb = nbands - 1; bb >= 0; --bb) {
        const Band t = band_info(d, n, L, bb);
        const int64_t sz = (d == 2) ? (int64_t)t.nj * t.nj : t.nj;
        if (s >= t.off && s < t.off + sz) {
            b = bb;
            Bo = t;
            break;
        }
    }
    const int rl = (int)(s - Bo.off);
    const int l0 = (d == 2) ? rl / Bo.nj : 0, l1 = (d == 2) ? rl % Bo.nj : rl;
    const int njb = Bo.nj;
    const T* vp = vals + op.row_ptr[s];
    const unsigned long long* dp = desc + s * op.nb;
    for (int k = 0; k < op.nb; ++k) {
        const unsigned long long w = dp[k];
        if (w == 0ull) break;
        const int b2 = (int)(w >> BLK_B2_SHIFT);
        int W0, W1, f0p, f1p;
        if (d == 2) {
            W0 = (int)(w & 0x3FFF);
            W1 = (int)((w >> 14) & 0x3FFF);
            f0p = (int)((w >> 28) & 0x3FFF);
            f1p = (int)((w >> 42) & 0x3FFF);
        } else {
            W0 = 1;
            W1 = (int)(w & 0xFFFFFFF);
            f0p = 0;
            f1p = (int)((w >> 28) & 0xFFFFFFF);
        }
        int kk = 0;
        for (int b3 = 0; b3 < b; ++b3) kk += block_kept(d, n, L, op.gap, b2, b3) ? 1 : 0;
        const Band B2 = band_info(d, n, L, b2);
        const int nj = B2.nj, tot = W0 * W1;
        const int rowstep = (d == 2) ? nj : 0;
        for (int i = lane; i < tot; i += 32) {
            const int a = i / W1, c = i - a * W1;
            int ra = f0p + a, cb = f1p + c;
            ra -= (ra >= nj) ? nj : 0;
            cb -= (cb >= nj) ? nj : 0;
            const int64_t lam = B2.off + (int64_t)ra * rowstep + cb;
            const unsigned long long w2 = desc[lam * op.nb + kk];
            int V0, V1, g0p, g1p;
            if (d == 2) {
                V0 = (int)(w2 & 0x3FFF);
                V1 = (int)((w2 >> 14) & 0x3FFF);
                g0p = (int)((w2 >> 28) & 0x3FFF);
                g1p = (int)((w2 >> 42) & 0x3FFF);
            } else {
                V0 = 1;
                V1 = (int)(w2 & 0xFFFFFFF);
                g0p = 0;
                g1p = (int)((w2 >> 28) & 0xFFFFFFF);
            }
            int a2 = l0 - g0p, c2 = l1 - g1p;
            a2 += (a2 < 0) ? njb : 0;
            c2 += (c2 < 0) ? njb : 0;
            if (w2 == 0ull || (int)(w2 >> BLK_B2_SHIFT) != b || a2 >= V0 || c2 >= V1) {
                flag_error(op.err, ERR_INDEX);
                continue;
            }
            valsT[op.row_ptr[lam] + boff[lam * op.nb + kk] + (int64_t)a2 * V1 + c2] = vp[i];
        }
        vp += tot;
    }
}

// One right-hand side (the solver's products).  LPR lanes per stored row (8, 16 or 32), so
// that with many rows the per-block set-up is shared by several rows of a warp and a block's
// last step wastes fewer lanes, while few rows still fill the device.  Lane t of a row takes
// entries t, t + LPR, ... of each kept column block (a W0 x W1 rectangle of translates,
// row-major), described by k_block_desc.  The rectangle coordinates advance by the fixed step
// LPR = qa * W1 + rb without divisions and wrap around
// the torus with one conditional subtraction (W0, W1 <= nj); column indices are 32-bit
// (N < 2^31).  Entries are taken four at a time so that four value and four x loads are in
// flight.
// TR = 0: y[s] = sum_e v_e x[col_e] - sub[s] (sub optional);
// TR = 1: y[col_e] += v_e x[s] (atomics into a zeroed y).
template <typename TV, typename TA, bool SQ, int TR, int LPR>
__global__ void __launch_bounds__(256) k_apply1(const __grid_constant__ OpDev<TA> op,
                                                const unsigned long long* __restrict__ desc,
                                                const TV* __restrict__ vals, const TA* __restrict__ x,
                                                TA* __restrict__ y, const TA* __restrict__ sub)
{
    static_assert(LPR == 8 || LPR == 16 || LPR == 32, "LPR");
    const int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / LPR;
    const int t = threadIdx.x & (LPR - 1);
    const bool live = s < op.N;
    const int d = op.d, n = op.n, L = op.L;
    TA acc = TA(0);
    if (live) {
        const TA xs = TR ? x[s] : TA(0);
        const TV* vp = vals + op.row_ptr[s];
        const unsigned long long* dp = desc + s * op.nb;
        for (int k = 0; k < op.nb; ++k) {
            const unsigned long long w = dp[k];
            if (w == 0ull) break;
            const int b2 = (int)(w >> BLK_B2_SHIFT);
            int W0, W1, f0p, f1p;
            if (d == 2) {
                W0 = (int)(w & 0x3FFF);
                W1 = (int)((w >> 14) & 0x3FFF);
                f0p = (int)((w >> 28) & 0x3FFF);
                f1p = (int)((w >> 42) & 0x3FFF);
            } else {
                W0 = 1;
                W1 = (int)(w & 0xFFFFFFF);
                f0p = 0;
                f1p = (int)((w >> 28) & 0xFFFFFFF);
            }
            const Band B2 = band_info(d, n, L, b2);
            const int nj = B2.nj, tot = W0 * W1;
            const int rowstep = (d == 2) ? nj : 0;
            const int off = (int)B2.off;
            int qa = 0, rb = LPR, a = 0, c = t;
            if (W1 < LPR) {
                qa = LPR / W1;
                rb = LPR - qa * W1;
                a = t / W1;
                c = t - a * W1;
            }
            for (int i0 = t; i0 < tot; i0 += 4 * LPR) {
                int col[4];
                TA v[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    int ra = f0p + a, cb = f1p + c;
                    ra -= (ra >= nj) ? nj : 0;
                    cb -= (cb >= nj) ? nj : 0;
                    col[u] = off + ra * rowstep + cb;
                    c += rb;
                    a += qa;
                    if (c >= W1) {
                        c -= W1;
                        ++a;
                    }
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int i = i0 + LPR * u;
                    v[u] = (i < tot) ? to_acc<TA, TV>(vp[i]) : TA(0);
                    if (SQ) v[u] *= v[u];
                }
                if (!TR) {
                    TA xv[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) xv[u] = (i0 + LPR * u < tot) ? x[col[u]] : TA(0);
#pragma unroll
                    for (int u = 0; u < 4; ++u) acc = fma(v[u], xv[u], acc);
                } else {
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        if (i0 + LPR * u < tot) atomicAdd(y + col[u], v[u] * xs);
                }
            }
            vp += tot;
        }
    }
    if (!TR) {
#pragma unroll
        for (int o = LPR / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (live && t == 0) y[s] = sub ? acc - sub[s] : acc;
    }
}

// y = S x for row-stored S (paper order), one warp per stored row.  The warp's lanes are
// (entry slot, group of 4 right-hand sides): LPE = NR/4 lanes read one entry's NR values of x
// as float4s (contiguous), 32/LPE entries per step; partial sums are reduced across entry
// slots with warp shuffles and the LPE lanes of slot 0 write y.  Requires x, y 16-byte
// aligned with ldx, ldy multiples of 4 (else k_apply is used).
template <typename TV, int NR>
__global__ void __launch_bounds__(256) k_apply_vec(const __grid_constant__ OpDev<float> op, const TV* __restrict__ vals,
                                                   const float* __restrict__ x, int ldx, float* __restrict__ y,
                                                   int ldy, int c0)
{
    static_assert(NR % 4 == 0 && NR <= 32, "NR");
    constexpr int LPE = NR / 4;        // lanes per entry
    constexpr int EPS = 32 / LPE;      // entries per step
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int slot = lane / LPE, quad = lane - slot * LPE;
    const int64_t s = warp;
    if (s >= op.N) return;
    const int d = op.d, n = op.n, L = op.L;
    int b = 0;
    Band Bo = band_info(d, n, L, 0);
    for (int bb = op.nb - 1; bb >= 0; --bb) {
        const Band t = band_info(d, n, L, bb);
        const int64_t sz = (d == 2) ? (int64_t)t.nj * t.nj : t.nj;
        if (s >= t.off && s < t.off + sz) {
            b = bb;
            Bo = t;
            break;
        }
    }
    const int rl = (int)(s - Bo.off);
    const int lg = log2i(Bo.nj);
    const int l0 = (d == 2) ? (rl >> lg) : 0, l1 = (d == 2) ? (rl & (Bo.nj - 1)) : rl;
    const int dense = op.gap < 0;
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    int64_t pos = op.row_ptr[s];
    const float* xq = x + c0 + 4 * quad;
    for (int b2 = 0; b2 < op.nb; ++b2) {
        if (!block_kept(d, n, L, op.gap, b, b2)) continue;
        const Band B2 = band_info(d, n, L, b2);
        int f0 = 0, W0 = 1, f1, W1;
        stencil(Bo.j, Bo.e1, l1, B2.j, B2.e1, op.r, op.Lf, n, dense, &f1, &W1);
        if (d == 2) stencil(Bo.j, Bo.e0, l0, B2.j, B2.e0, op.r, op.Lf, n, dense, &f0, &W0);
        const int nj = B2.nj, njm = nj - 1, tot = W0 * W1;
        const int64_t rowstride = (d == 2) ? nj : 0;
        int a = slot / W1, bb = slot - (slot / W1) * W1;
        const int da = EPS / W1, db = EPS - da * W1;
        for (int idx = slot; idx < tot; idx += EPS) {
            const int64_t col = B2.off + (int64_t)((f0 + a) & njm) * rowstride + ((f1 + bb) & njm);
            const float v = to_acc<float, TV>(vals[pos + idx]);
            const float4 xv = *reinterpret_cast<const float4*>(xq + col * ldx);
            acc.x = fmaf(v, xv.x, acc.x);
            acc.y = fmaf(v, xv.y, acc.y);
            acc.z = fmaf(v, xv.z, acc.z);
            acc.w = fmaf(v, xv.w, acc.w);
            a += da;
            bb += db;
            if (bb >= W1) {
                bb -= W1;
                ++a;
            }
        }
        pos += tot;
    }
#pragma unroll
    for (int o = LPE; o < 32; o <<= 1) {
        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
        acc.z += __shfl_xor_sync(0xffffffffu, acc.z, o);
        acc.w += __shfl_xor_sync(0xffffffffu, acc.w, o);
    }
    if (slot == 0) *reinterpret_cast<float4*>(y + s * ldy + c0 + 4 * quad) = acc;
}

// ------------------------------------------------------------------------------------------
// Apply on tensor cores: y = S x for 16 right-hand sides, BF16 S, FP32 accumulation.
// A CTA (4 warps) owns a tile of 16 stored rows of one band with the same l0 and consecutive
// l1.  For each kept column band b2 and each stencil row a (warps take a's in turn), the 16
// rows' entries form a banded 16 x K block A (row i holds its W1(i) values at column offset
// o_i) and the matching K x 16 slab of x (row f0 + a of band b2, columns u .. u + K - 1 mod
// nj2) is B; mma.sync m16n8k16 (BF16 inputs, FP32 accumulate) adds A B to the warp's 16 x 16
// accumulator.  x is split once per call into hi + lo BF16 parts (k_split_x; two products) so
// that the only rounding beyond FP32 is the BF16 storage of S.  Warps' partial sums are reduced
// in shared memory.
// ------------------------------------------------------------------------------------------
struct TcApply {
    int d, n, L, Lf, r, gap, nb;
    int64_t N;
    const int64_t* row_ptr;
    int tile_off[MAXB + 1];  // first tile of band b (tiles: l0 x ceil(nj / 16))
};

__device__ __forceinline__ unsigned pack_bf16(float lo, float hi)
{
    const __nv_bfloat16 a = __float2bfloat16_rn(lo), b = __float2bfloat16_rn(hi);
    return (unsigned)__bfloat16_as_ushort(a) | ((unsigned)__bfloat16_as_ushort(b) << 16);
}

__device__ __forceinline__ void mma_bf16_16816(float (&c)[4], unsigned a0, unsigned a1, unsigned a2, unsigned a3,
                                               unsigned b0, unsigned b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// x (16 right-hand sides from column c0) split once per call into BF16 parts hi + lo (x to
// ~2^-16 relative), packed per element as hi | lo << 16: xs[i * 16 + c].
__global__ void k_split_x(const float* __restrict__ x, int ldx, int c0, int64_t N, unsigned* __restrict__ xs)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N * 16) return;
    const float v = x[(i >> 4) * ldx + c0 + (i & 15)];
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    const __nv_bfloat16 l = __float2bfloat16_rn(v - __bfloat162float(h));
    xs[i] = (unsigned)__bfloat16_as_ushort(h) | ((unsigned)__bfloat16_as_ushort(l) << 16);
}

__global__ void __launch_bounds__(128) k_apply_tc(const __grid_constant__ TcApply tp,
                                                  const __nv_bfloat16* __restrict__ vals,
                                                  const unsigned* __restrict__ xs, float* __restrict__ y, int ldy,
                                                  int c0)
{
    __shared__ int64_t rbase[16];          // row_ptr of the tile's rows
    __shared__ int boff[16][MAXB];         // block offsets within each row
    __shared__ int f1s[16][MAXB], w1s[16][MAXB];
    __shared__ int f0s[MAXB], w0s[MAXB];
    __shared__ float red[4][16][17];
    const int d = tp.d, n = tp.n, L = tp.L;
    const int tile = blockIdx.x;
    int b = 0;
    while (b + 1 < tp.nb && tile >= tp.tile_off[b + 1]) ++b;
    const Band Bo = band_info(d, n, L, b);
    const int nt1 = (Bo.nj + 15) >> 4;
    const int tl = tile - tp.tile_off[b];
    const int l0 = (d == 2) ? tl / nt1 : 0;
    const int l1base = (tl - l0 * nt1) * 16;
    const int nvalid = min(16, Bo.nj - l1base);
    const int dense = tp.gap < 0;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // per-row stencils (all threads over (row, block) pairs), then block offsets (thread i: row i)
    for (int e = threadIdx.x; e < 16 * tp.nb; e += blockDim.x) {
        const int i = e / tp.nb, b2 = e - i * tp.nb;
        const int l1 = l1base + min(i, nvalid - 1);
        if (!block_kept(d, n, L, tp.gap, b, b2)) {
            w1s[i][b2] = 0;
            if (i == 0) w0s[b2] = 0;
            continue;
        }
        const Band B2 = band_info(d, n, L, b2);
        int f0 = 0, W0 = 1, f1, W1;
        stencil(Bo.j, Bo.e1, l1, B2.j, B2.e1, tp.r, tp.Lf, n, dense, &f1, &W1);
        if (d == 2 && i == 0) stencil(Bo.j, Bo.e0, l0, B2.j, B2.e0, tp.r, tp.Lf, n, dense, &f0, &W0);
        f1s[i][b2] = f1;
        w1s[i][b2] = W1;
        if (i == 0) {
            f0s[b2] = f0;
            w0s[b2] = W0;
        }
    }
    __syncthreads();
    if (threadIdx.x < 16) {
        const int i = threadIdx.x;
        const int l1 = l1base + min(i, nvalid - 1);
        const int64_t s = Bo.off + (int64_t)l0 * ((d == 2) ? Bo.nj : 0) + l1;
        rbase[i] = tp.row_ptr[s];
        int acc = 0;
        for (int b2 = 0; b2 < tp.nb; ++b2) {
            boff[i][b2] = acc;
            acc += w0s[b2] * w1s[i][b2];
        }
    }
    __syncthreads();
    const int g = lane >> 2, q = lane & 3;
    float acc0[4] = {0.f, 0.f, 0.f, 0.f}, acc1[4] = {0.f, 0.f, 0.f, 0.f};  // n-tiles 0 (rhs 0..7), 1 (8..15)
    const bool vg = g < nvalid, vg8 = g + 8 < nvalid;
    for (int b2 = 0; b2 < tp.nb; ++b2) {
        if (w1s[0][b2] == 0) continue;
        const Band B2 = band_info(d, n, L, b2);
        const int nj2 = B2.nj, m2 = nj2 - 1;
        const int W0 = w0s[b2], f0 = f0s[b2];
        // union of the rows' windows on axis 1 (first rows start first: stencils are monotone)
        const int u = f1s[0][b2];
        int K = 0;
        for (int i = 0; i < nvalid; ++i) K = max(K, f1s[i][b2] + w1s[i][b2] - u);
        const int Wg = w1s[g][b2], Wg8 = w1s[g + 8][b2];
        const int og = f1s[g][b2] - u, og8 = f1s[g + 8][b2] - u;
        const __nv_bfloat16* rg = vals + rbase[g] + boff[g][b2];
        const __nv_bfloat16* rg8 = vals + rbase[g + 8] + boff[g + 8][b2];
        for (int a = warp; a < W0; a += 4) {
            const int64_t xrow = B2.off + (int64_t)((f0 + a) & m2) * ((d == 2) ? nj2 : 0);
            const __nv_bfloat16* ag = rg + a * Wg - og;
            const __nv_bfloat16* ag8 = rg8 + a * Wg8 - og8;
#pragma unroll 2
            for (int kc = 0; kc < K; kc += 16) {
                unsigned A[4];
#pragma unroll
                for (int h = 0; h < 2; ++h) {        // columns 2q + 8h, 2q + 8h + 1
                    const int k0 = kc + 2 * q + 8 * h, k1 = k0 + 1;
                    const bool g0ok = vg && k0 >= og && k0 < og + Wg, g1ok = vg && k1 >= og && k1 < og + Wg;
                    const bool h0ok = vg8 && k0 >= og8 && k0 < og8 + Wg8, h1ok = vg8 && k1 >= og8 && k1 < og8 + Wg8;
                    unsigned short x0 = 0, x1 = 0, z0 = 0, z1 = 0;
                    if (g0ok) x0 = __bfloat16_as_ushort(ag[k0]);
                    if (g1ok) x1 = __bfloat16_as_ushort(ag[k1]);
                    if (h0ok) z0 = __bfloat16_as_ushort(ag8[k0]);
                    if (h1ok) z1 = __bfloat16_as_ushort(ag8[k1]);
                    A[2 * h] = (unsigned)x0 | ((unsigned)x1 << 16);
                    A[2 * h + 1] = (unsigned)z0 | ((unsigned)z1 << 16);
                }
#pragma unroll
                for (int nt = 0; nt < 2; ++nt) {
                    unsigned xp[4];  // (hi, lo) of x at chunk columns 2q, 2q+1, 2q+8, 2q+9
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        const int kk = kc + 2 * q + (t & 1) + 8 * (t >> 1);
                        xp[t] = (kk < K) ? __ldg(xs + (xrow + ((u + kk) & m2)) * 16 + nt * 8 + g) : 0u;
                    }
                    const unsigned bh0 = __byte_perm(xp[0], xp[1], 0x5410), bh1 = __byte_perm(xp[2], xp[3], 0x5410);
                    const unsigned bl0 = __byte_perm(xp[0], xp[1], 0x7632), bl1 = __byte_perm(xp[2], xp[3], 0x7632);
                    float(&acc)[4] = nt ? acc1 : acc0;
                    mma_bf16_16816(acc, A[0], A[1], A[2], A[3], bh0, bh1);
                    mma_bf16_16816(acc, A[0], A[1], A[2], A[3], bl0, bl1);
                }
            }
        }
    }
    // C fragments: (row g, cols 2q, 2q+1), (row g + 8, cols 2q, 2q+1) per n-tile
    red[warp][g][2 * q] = acc0[0];
    red[warp][g][2 * q + 1] = acc0[1];
    red[warp][g + 8][2 * q] = acc0[2];
    red[warp][g + 8][2 * q + 1] = acc0[3];
    red[warp][g][8 + 2 * q] = acc1[0];
    red[warp][g][8 + 2 * q + 1] = acc1[1];
    red[warp][g + 8][8 + 2 * q] = acc1[2];
    red[warp][g + 8][8 + 2 * q + 1] = acc1[3];
    __syncthreads();
    for (int e = threadIdx.x; e < 16 * 16; e += blockDim.x) {
        const int i = e >> 4, c = e & 15;
        if (i < nvalid) {
            const float v = red[0][i][c] + red[1][i][c] + red[2][i][c] + red[3][i][c];
            const int64_t s = Bo.off + (int64_t)l0 * ((d == 2) ? Bo.nj : 0) + l1base + i;
            y[s * ldy + c0 + c] = v;
        }
    }
}

template <typename TA>
__global__ void k_zero_rows(TA* y, int64_t N, int ldy, int c0, int nr)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < N * nr) y[(i / nr) * ldy + c0 + (i % nr)] = TA(0);
}

// ------------------------------------------------------------------------------------------
// Deblurring in the wavelet domain (Section 4.3; FISTA-W / FISTA-WP of the appendix on
// deblurring algorithms): the vector kernels of one iteration and of the power iteration
// that bounds the step.  S = diag(sigma) is the preconditioner (identity when sigma is null).
// ------------------------------------------------------------------------------------------
template <typename T>
__global__ void k_fill_vec(T* __restrict__ v, int64_t N, T val)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) v[i] = val;
}

// v[i] *= sqrt(sigma[i])
template <typename T>
__global__ void k_scale_sqrt(T* __restrict__ v, const T* __restrict__ sigma, int64_t N)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) v[i] *= sqrt(sigma[i]);
}

// out[0] += sum_i v[i]^2, FP64 block partial sums (out zeroed by the caller)
template <typename T>
__global__ void __launch_bounds__(256) k_norm2(const T* __restrict__ v, int64_t N, double* __restrict__ out)
{
    __shared__ double part[8];
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        acc += (double)v[i] * (double)v[i];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
        atomicAdd(out, t);
    }
}

// u = g / sqrt(nrm2[0]) (zero when the norm is zero)
template <typename T>
__global__ void k_normalize(T* __restrict__ u, const T* __restrict__ g, int64_t N, const double* __restrict__ nrm2)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const double s = nrm2[0];
    if (i < N) u[i] = (s > 0.0) ? (T)((double)g[i] / sqrt(s)) : T(0);
}

// One FISTA update from the gradient g = Theta^T (Theta y - z0):
//   a = y - tau s g,  z' = soft(a, tau s w),  y = z' + beta (z' - z),  z = z'
// with s = sigma[i] (1 without preconditioner).
template <typename T>
__global__ void k_fista_step(T* __restrict__ z, T* __restrict__ y, const T* __restrict__ g, const T* __restrict__ w,
                             const T* __restrict__ sigma, int64_t N, T tau, T beta)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const T ts = sigma ? tau * sigma[i] : tau;
    const T a = y[i] - ts * g[i];
    const T t = ts * w[i];
    const T zn = (a > t) ? a - t : (a < -t) ? a + t : T(0);
    y[i] = zn + beta * (zn - z[i]);
    z[i] = zn;
}

}  // namespace pcw
