// Group kernel: one CTA chases K consecutive sweeps of a bandwidth-reduction
// stage together (arXiv 2510.12705, Section III: Algorithm 1 schedule,
// Algorithm 2 row-bulge; the sweeps of a group are the paper's "max blocks"
// unrolled into one block).
//
// Geometry (stage bw -> bw' = bw - d, group g = sweeps R0 = gK .. R0+K-1,
// step s, origin c = R0 + bw' + s bw; window coordinates I = row - c,
// X = column - c).  Member j works at c + j: its right reflector comes from
// row I_j = j - bw (j - bw' at s = 0), columns j .. j+m-1, and is applied to
// rows I_j+1 .. j+m-1; its left reflector comes from column j, rows
// j .. j+m-1, and is applied to columns j+1 .. j+m-1+bw.  The union of the
// members' footprints is held in shared memory as
//   V  columns X in [0, K+d), rows I in [-bw, K+d)   (odd pitch PV)
//   H  columns X in [K+d, bw), rows I in [0, K+d)    (odd pitch PH)
//   columns X in [bw, bw+K+d), rows I in [0, K+d): the next step's first
//      rows (the carried block), kept in V's first K+d physical rows.
//
// Per step: wait until group g-1 completed step s; load the window except the
// carried block and the tail columns [bw-K, bw); phase U: every member's right
// reflector, applied to the rows above c; then phase L: per member the right
// reflector on the rows at or below c, then the left reflector.  Members work
// step by step, not sweep by sweep: member j+1's left reflector at step s runs
// before member j's right reflector at step s+1; the two transform disjoint
// generating vectors and a common block that each transforms whole, so they
// commute (equal in exact arithmetic).  Across groups the order of every
// conflicting pair is the sequential one.  3K + d <= bw keeps group g-2's step
// s+2 out of group g's window.
//
// The two phases run as three pipelines of warps, so that the chains of
// reflector generations do not wait for the bulk of the updates (the rows
// above c and the rows at or below c are disjoint, so the phases overlap):
//   warp 0       builds the right reflectors in member order and applies each
//                one itself to the rows the later members build theirs from
//                (rows I_{j+1} .. I_{ka-1}), then publishes it (a shared-
//                memory flag, release / acquire at CTA scope);
//   warps 1..NT  the near team: per member, as soon as its right reflector is
//                published, the right reflector on the rows at or below c,
//                the left reflector (warp 1) and its update of the columns
//                X < K+d, with the team's named barrier; this part of the
//                window is complete after the wait above;
//   the rest     the far team: each right reflector, as published, on the
//                rows I_last+1 .. -1 (each row always in the same thread);
//                then the rows above c go back to the band and "upper part of
//                step s done" is published; then the wait until group g-1 did
//                the upper part of step s+1 (it writes the tail columns), the
//                load of the tail and the next carried block, and each left
//                reflector, as published, on the columns X >= K+d (each column
//                always in the same thread).
// Then all warps store the rows at or below c and publish "step s complete".
// Every element sees the same transformations in the same order as in the
// plain member-by-member program; the small updates on the two chains use
// four lanes per row or column (a fixed summation order).  The host model in
// tests/test_group_protocol.py checks the schedule element by element.
#pragma once

#include "bb_device.cuh"

namespace bb {

// members per group on a stage (0: the stage runs the per-sweep kernel)
__host__ __device__ __forceinline__ int group_members(int bw, int d, int K)
{
    const int lim = (bw - d) / 3;
    return K < lim ? K : lim;
}

// shared-memory elements (compute type) of the group kernel for one problem
__host__ __device__ __forceinline__ int group_pv(int bw, int d, int K) { return (bw + K + d) | 1; }
__host__ __device__ __forceinline__ int group_ph(int d, int K) { return (K + d) | 1; }
__host__ __device__ __forceinline__ int group_small_elems(int kmax, int maxm)
{
    // vR[kmax][maxm], tbR[kmax][4], vL[kmax][maxm], tbL[kmax][4], xb[maxm+1], 64 spare, 16-byte rounding
    return ((2 * kmax * maxm + 8 * kmax + (maxm + 1) + 64) + 3) & ~3;
}
// warps of the near team (warps 1 .. NT; warp 0 leads phase U, the rest are
// far warps); the kernel runs with at least four warps
__host__ __device__ __forceinline__ int group_near_warps(int nw) { return nw - 2 < 3 ? nw - 2 : 3; }
__host__ __device__ __forceinline__ int group_window_elems(int bw, int d, int K)
{
    return (K + d) * group_pv(bw, d, K) + (bw - K - d) * group_ph(d, K);
}

// Right reflector (v, tau) on window rows [r_lo, r_hi] of columns [j, j+m):
// element (I, X) at V[X * PV + I + bw].  Lanes 0-15 take 16 consecutive rows
// and columns j .. j+HA-1 (and j+2HA), lanes 16-31 the same rows and columns
// j+HA .. j+2HA-1; one shuffle combines the two halves of each dot product.
// Only warps [w0, w1) take part (w1 <= 0: up to the last warp).
template <typename T, int MAXM>
__device__ __forceinline__ void group_apply_right(T* V, int PV, int bw, int j, int m, int r_lo,
                                                  int r_hi, const T* v, T tau, int w0 = 0, int w1 = 0)
{
    constexpr int HA = (MAXM - 1) / 2;
    constexpr bool EXTRA = MAXM == 2 * HA + 1;
    const int lane = threadIdx.x & 31;
    const int warp = (threadIdx.x >> 5) - w0, nw = (w1 > 0 ? w1 : (int)(blockDim.x >> 5)) - w0;
    if (warp < 0 || warp >= nw) return;
    const int half = lane >> 4, l = lane & 15;
    const int t0 = half * HA;
    const int nrows = r_hi - r_lo + 1;
    // loads from clamped, always valid addresses (no branch per entry); v is
    // zero beyond m, so the extra terms vanish; only the stores are guarded
    for (int base = warp * 16; base < nrows; base += nw * 16) {
        const bool act = base + l < nrows;
        const int r = r_lo + (act ? base + l : nrows - 1) + bw;
        T a[HA];
        T w = (T)0;
#pragma unroll
        for (int i = 0; i < HA; ++i) {
            const int t = t0 + i < m ? t0 + i : m - 1;
            a[i] = V[(j + t) * PV + r];
            w = fma(a[i], v[t0 + i], w);
        }
        T a2 = (T)0;
        if (EXTRA && half == 0) {
            a2 = V[(j + (2 * HA < m ? 2 * HA : m - 1)) * PV + r];
            w = fma(a2, v[2 * HA], w);
        }
        w += __shfl_xor_sync(FULL, w, 16);
        const T tw = tau * w;
        if (act) {
#pragma unroll
            for (int i = 0; i < HA; ++i)
                if (t0 + i < m) V[(j + t0 + i) * PV + r] = fma(-tw, v[t0 + i], a[i]);
            if (EXTRA && half == 0 && 2 * HA < m) V[(j + 2 * HA) * PV + r] = fma(-tw, v[2 * HA], a2);
        }
    }
}

// Window column X as a pointer to its row I = 0 (valid rows as above).
template <typename T>
struct GroupCols {
    T* V;
    T* H;
    int PV, PH, bw, KD;   // KD = K + d
    __device__ __forceinline__ T* operator()(int X) const
    {
        if (X < KD) return V + X * PV + bw;
        if (X < bw) return H + (X - KD) * PH;
        return V + (X - bw) * PV;
    }
};

// Left reflector (v, tau) on rows [j, j+m) of window columns [x_lo, x_hi]:
// lanes 0-15 take 16 consecutive columns and rows j .. j+HA-1 (and j+2HA),
// lanes 16-31 the same columns and rows j+HA .. j+2HA-1.
template <typename T, int MAXM>
__device__ __forceinline__ void group_apply_left(const GroupCols<T>& col, int j, int m, int x_lo,
                                                 int x_hi, const T* v, T tau, int w0 = 0, int w1 = 0)
{
    constexpr int HA = (MAXM - 1) / 2;
    constexpr bool EXTRA = MAXM == 2 * HA + 1;
    const int lane = threadIdx.x & 31;
    const int warp = (threadIdx.x >> 5) - w0, nw = (w1 > 0 ? w1 : (int)(blockDim.x >> 5)) - w0;
    if (warp < 0 || warp >= nw) return;
    const int half = lane >> 4, l = lane & 15;
    const int t0 = half * HA;
    const int ncols = x_hi - x_lo + 1;
    for (int base = warp * 16; base < ncols; base += nw * 16) {
        const bool act = base + l < ncols;
        T* p = col(x_lo + (act ? base + l : ncols - 1)) + j;
        T a[HA];
        T w = (T)0;
#pragma unroll
        for (int i = 0; i < HA; ++i) {
            a[i] = p[t0 + i < m ? t0 + i : m - 1];
            w = fma(a[i], v[t0 + i], w);
        }
        T a2 = (T)0;
        if (EXTRA && half == 0) {
            a2 = p[2 * HA < m ? 2 * HA : m - 1];
            w = fma(a2, v[2 * HA], w);
        }
        w += __shfl_xor_sync(FULL, w, 16);
        const T tw = tau * w;
        if (act) {
#pragma unroll
            for (int i = 0; i < HA; ++i)
                if (t0 + i < m) p[t0 + i] = fma(-tw, v[t0 + i], a[i]);
            if (EXTRA && half == 0 && 2 * HA < m) p[2 * HA] = fma(-tw, v[2 * HA], a2);
        }
    }
}

// Small updates on the reflector chain, four lanes per row (column): lane q
// of a quad takes the reflector entries q, q+4, q+8, ...; two shuffles combine
// the partial dot products (a fixed order, whatever the warp count).  Short
// per-lane chains and all 32 lanes busy matter here: these updates sit
// between two reflector generations.  Warps [w0, w1) take part.
template <typename T, int MAXM>
__device__ __forceinline__ void quad_apply_right(T* V, int PV, int bw, int j, int m, int r_lo, int r_hi,
                                                 const T* v, T tau, int w0, int w1)
{
    constexpr int NQ = (MAXM + 3) / 4;
    const int lane = threadIdx.x & 31;
    const int warp = (threadIdx.x >> 5) - w0, nw = w1 - w0;
    if (warp < 0 || warp >= nw) return;
    const int q = lane & 3, rl = lane >> 2;
    const int nrows = r_hi - r_lo + 1;
    for (int base = warp * 8; base < nrows; base += nw * 8) {
        const bool act = base + rl < nrows;
        const int r = r_lo + (act ? base + rl : nrows - 1) + bw;
        T a[NQ];
        T w = (T)0;
#pragma unroll
        for (int i = 0; i < NQ; ++i) {
            const int t0 = q + 4 * i;
            a[i] = V[(j + (t0 < m ? t0 : m - 1)) * PV + r];
            if (t0 < MAXM) w = fma(a[i], v[t0], w);
        }
        w += __shfl_xor_sync(FULL, w, 1);
        w += __shfl_xor_sync(FULL, w, 2);
        const T tw = tau * w;
        if (act) {
#pragma unroll
            for (int i = 0; i < NQ; ++i) {
                const int t0 = q + 4 * i;
                if (t0 < m) V[(j + t0) * PV + r] = fma(-tw, v[t0], a[i]);
            }
        }
    }
}

template <typename T, int MAXM>
__device__ __forceinline__ void quad_apply_left(const GroupCols<T>& col, int j, int m, int x_lo, int x_hi,
                                                const T* v, T tau, int w0, int w1)
{
    constexpr int NQ = (MAXM + 3) / 4;
    const int lane = threadIdx.x & 31;
    const int warp = (threadIdx.x >> 5) - w0, nw = w1 - w0;
    if (warp < 0 || warp >= nw) return;
    const int q = lane & 3, cl = lane >> 2;
    const int ncols = x_hi - x_lo + 1;
    for (int base = warp * 8; base < ncols; base += nw * 8) {
        const bool act = base + cl < ncols;
        T* p = col(x_lo + (act ? base + cl : ncols - 1)) + j;
        T a[NQ];
        T w = (T)0;
#pragma unroll
        for (int i = 0; i < NQ; ++i) {
            const int t0 = q + 4 * i;
            a[i] = p[t0 < m ? t0 : m - 1];
            if (t0 < MAXM) w = fma(a[i], v[t0], w);
        }
        w += __shfl_xor_sync(FULL, w, 1);
        w += __shfl_xor_sync(FULL, w, 2);
        const T tw = tau * w;
        if (act) {
#pragma unroll
            for (int i = 0; i < NQ; ++i) {
                const int t0 = q + 4 * i;
                if (t0 < m) p[t0] = fma(-tw, v[t0], a[i]);
            }
        }
    }
}

// Copy window columns [x_lo, x_hi] between the working band and shared
// memory (LOAD: band -> shared with cp.async; else shared -> band), one warp
// per column, rows rows(X) = [lo, hi] clipped to the matrix.  Element
// (c + I, c + X) of the band is at Wg[(c + X) * ldw + top - X + I].  Warps
// [w0, nw) take part (the others return at once).
template <typename TS, typename T, bool LOAD, typename Rows>
__device__ __forceinline__ void group_copy(TS* __restrict__ Wg, int ldw, int top, int n, int c,
                                           int x_lo, int x_hi, const GroupCols<T>& col, Rows rows,
                                           int w0 = 0)
{
    const int lane = threadIdx.x & 31, warp = (threadIdx.x >> 5) - w0, nw = (blockDim.x >> 5) - w0;
    if (warp < 0) return;
    x_hi = min(x_hi, n - 1 - c);
    for (int X = x_lo + warp; X <= x_hi; X += nw) {
        int lo, hi;
        rows(X, lo, hi);
        lo = max(lo, -c);
        hi = min(hi, n - 1 - c);
        T* sp = col(X);
        TS* gp = Wg + (int64_t)(c + X) * ldw + (top - X);
        for (int I = lo + lane; I <= hi; I += 32) {
            if constexpr (LOAD) band_to_panel<TS, T>(sp + I, gp + I);
            else panel_to_band<TS, T>(gp + I, sp[I]);
        }
    }
}

// One lane waits until the shared-memory flag *p >= target (a producer warp of
// this CTA raises it with a release); bounded like wait_at_least: gives up
// (sets the error and abort words) after timeout_ns or when another CTA aborted.
__device__ __forceinline__ bool wait_flag(const int* p, int target, Header* hdr,
                                          unsigned long long timeout_ns)
{
    if (ld_relaxed_shared(p) >= target) { (void)ld_acquire_shared(p); return true; }
    const unsigned long long t0 = global_ns();
    for (int it = 1;; ++it) {
        if (it > 16) __nanosleep(20);
        if (ld_relaxed_shared(p) >= target) { (void)ld_acquire_shared(p); return true; }
        if ((it & 63) == 0) {
            if (ld_relaxed(&hdr->abort)) return false;
            if (global_ns() - t0 > timeout_ns) {
                atomicOr(&hdr->err, 1 << 4 /* BB_ERR_TIMEOUT */);
                atomicExch(&hdr->abort, 1);
                return false;
            }
        }
    }
}

// The whole warp waits on a flag: lane 0 acquires, the shuffle and __syncwarp
// order the other lanes' reads after it.
__device__ __forceinline__ bool warp_wait_flag(const int* p, int target, Header* hdr,
                                               unsigned long long timeout_ns)
{
    int ok = 1;
    if ((threadIdx.x & 31) == 0) ok = (int)wait_flag(p, target, hdr, timeout_ns);
    ok = __shfl_sync(FULL, ok, 0);
    __syncwarp();
    return ok != 0;
}

// The warp's shared-memory writes so far, then the flag (release).
__device__ __forceinline__ void warp_publish(int* p, int v)
{
    __syncwarp();
    if ((threadIdx.x & 31) == 0) st_release_shared(p, v);
}

template <typename TS, typename T, int MAXM>
__global__ void __launch_bounds__(384, 2) group_kernel(Launch L)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int KMAX = L.gK;
    T* const vR = (T*)smem_raw;                 // KMAX x MAXM right reflector vectors
    T* const tbR = vR + KMAX * MAXM;            // KMAX x {tau, beta, vs, -}
    T* const vL = tbR + KMAX * 4;               // KMAX x MAXM left reflector vectors
    T* const tbL = vL + KMAX * MAXM;            // KMAX x {tau, beta, vs, -}
    T* const xb = tbL + KMAX * 4;               // staged reflector input
    T* const V = (T*)smem_raw + group_small_elems(KMAX, MAXM);
    __shared__ int s_task[2];
    __shared__ int s_ok;        // W1 and the final wait (thread 0)
    __shared__ int s_ok2;       // W2 (first far thread)
    __shared__ int s_nfail;     // a flag wait of the near team gave up
    __shared__ int s_ffail;     // a flag wait of the far team gave up
    __shared__ int s_uflag;     // phase U: 128 s + (right reflectors published)
    __shared__ int s_lflag;     // phase L: 128 s + (left reflectors published)
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nw = blockDim.x >> 5;
    const int NT = group_near_warps(nw);
    const int stage = L.stage;
    const int base = stage * PROG_STAGE;
    const int ps = L.prog_stride;

    for (;;) {
        if (tid == 0) {
            int t = -1;
            if (!ld_relaxed(&L.hdr->abort)) t = atomicAdd(&L.hdr->claim, 1);
            if (t >= 0 && t < L.total_tasks) {
                s_task[0] = t % L.count;
                s_task[1] = t / L.count;
            } else {
                s_task[0] = -1;
            }
            s_uflag = 0;
            s_lflag = 0;
            s_nfail = 0;
            s_ffail = 0;
        }
        __syncthreads();
        const int q = s_task[0];
        if (q < 0) break;
        const int g = s_task[1];
        const Desc& D = desc_of(L, q);
        __syncthreads();
        if (stage >= D.nstages) continue;
        const int n = D.n;
        const int bw = stage_bw(D.b, L.tw, stage);
        const int d = stage_d(bw, L.tw);
        const int bwp = bw - d;
        const int K = group_members(bw, d, KMAX);
        if (K < 1) continue;
        const int nact = n - 1 - bwp;
        if (nact <= 0 || g >= (nact + K - 1) / K) continue;
        const int R0 = g * K;
        const int kk = min(K, nact - R0);
        const int S = sweep_steps(n, bw, d, R0);
        const int Sp = g > 0 ? sweep_steps(n, bw, d, R0 - K) : 0;
        const int KD = K + d;
        const int PV = group_pv(bw, d, K), PH = group_ph(d, K);
        const GroupCols<T> col{V, V + KD * PV, PV, PH, bw, KD};
        TS* const Wg = (TS*)L.wbase + D.w_off;
        const int ldw = D.ldw, top = D.top;
        int* const my = L.prog + D.prog_off + (int64_t)g * ps;
        const int* const pred = g > 0 ? my - ps : nullptr;
        const bool stall = (L.flags & BB_FLAG_INJECT_STALL) && stage == 0 && g == 0;
        bool ok = true;

        for (int s = 0; s < S && ok; ++s) {
            const int c = R0 + bwp + s * bw;
            const int vt = s == 0 ? bwp : bw;     // V column X starts at row max(0, X-d) - vt
            const int fb = 128 * s;               // flag values of this step (K <= 64)
            int ka = 0;                           // members active at this step (a prefix)
            while (ka < kk && s < sweep_steps(n, bw, d, R0 + ka)) ++ka;

            // ---- W1: group g-1 completed step s
            if (tid == 0) s_ok = (g == 0) ? 1 : (int)wait_at_least(pred, base + 2 * (s + 1), L.hdr, L.timeout_ns);
            __syncthreads();
            if (!s_ok) { ok = false; break; }
            // ---- LD1: V (without the carried rows) and H before the tail
            group_copy<TS, T, true>(Wg, ldw, top, n, c, 0, KD - 1, col, [&](int X, int& lo, int& hi) {
                lo = (s == 0) ? max(0, X - d) - vt : KD - bw;
                hi = min(K - 1, X) + d;
            });
            group_copy<TS, T, true>(Wg, ldw, top, n, c, KD, bw - (g > 0 ? K : 0) - 1, col,
                                    [&](int, int& lo, int& hi) { lo = 0; hi = KD - 1; });
            cp_async_wait_all();
            __syncthreads();

            // ---- phases U and L as three pipelines of warps (after LD1; the
            //      rows above c and the rows at or below c are disjoint):
            //   warp 0       the right reflectors in member order; it keeps the
            //                members' reflector rows I_1 .. I_last up to date
            //   warps 1..NT  per member: the right reflector on the rows >= c,
            //                the left reflector (warp 1), its near columns
            //   the rest     the right reflectors on the rows I_last+1 .. -1;
            //                ST1 and the half mark; W2; LD2; the left
            //                reflectors on the far columns
            // A flag wait is taken by one warp of a team and handed on by the
            // team's barrier, so a failed wait stops the whole team at once.
            const int Ilast = ka - 1 - vt;
            const int F0 = 1 + NT, nf = nw - F0;          // far warps [F0, nw)
            if (warp == 0) {
                for (int j = 0; j < ka; ++j) {
                    const int m = min(d + 1, n - (c + j));
                    const int Ij = j - vt;
                    T* vj = vR + j * MAXM;
                    T* tj = tbR + j * 4;
                    for (int t = lane; t < m; t += 32) xb[t] = V[(j + t) * PV + Ij + bw];
                    __syncwarp();
                    fast_reflector<T, MAXM>(m, xb, vj, tj);
                    __syncwarp();
                    if (L.refl) warp_store_reflector<T, MAXM>(L, n, bw, d, R0 + j, s, 0, m, vj, tj[0]);
                    for (int t = lane; t < m; t += 32) V[(j + t) * PV + Ij + bw] = t == 0 ? tj[1] : (T)0;
                    if (Ij + 1 <= Ilast)
                        quad_apply_right<T, MAXM>(V, PV, bw, j, m, Ij + 1, Ilast, vj, tj[0], 0, 1);
                    warp_publish(&s_uflag, fb + j + 1);
                }
            } else if (warp < F0) {
                for (int j = 0; j < ka; ++j) {
                    const int m = min(d + 1, n - (c + j));
                    const int jmax = min(n - 1 - c, j + m - 1 + bw);
                    if (warp == 1 && !warp_wait_flag(&s_uflag, fb + j + 1, L.hdr, L.timeout_ns) && lane == 0)
                        s_nfail = 1;
                    bar_sync_n(1, 32 * NT);
                    if (s_nfail) break;
                    quad_apply_right<T, MAXM>(V, PV, bw, j, m, 0, j + m - 1, vR + j * MAXM, tbR[j * 4], 1, F0);
                    bar_sync_n(1, 32 * NT);
                    T* vl = vL + j * MAXM;
                    T* tl = tbL + j * 4;
                    if (warp == 1) {
                        T* x = V + j * PV + bw + j;          // column j, rows j .. j+m-1
                        fast_reflector<T, MAXM>(m, x, vl, tl);
                        __syncwarp();
                        if (L.refl) warp_store_reflector<T, MAXM>(L, n, bw, d, R0 + j, s, 1, m, vl, tl[0]);
                        for (int t = lane; t < m; t += 32) x[t] = t == 0 ? tl[1] : (T)0;
                        warp_publish(&s_lflag, fb + j + 1);
                    }
                    bar_sync_n(1, 32 * NT);
                    const int xn = min(jmax, KD - 1);
                    if (j + 1 <= xn) quad_apply_left<T, MAXM>(col, j, m, j + 1, xn, vl, tl[0], 1, F0);
                    bar_sync_n(1, 32 * NT);
                }
            } else {
                const bool lead = warp == F0;                 // takes the far team's waits
                for (int j = 0; j < ka; ++j) {
                    if (lead && !warp_wait_flag(&s_uflag, fb + j + 1, L.hdr, L.timeout_ns) && lane == 0)
                        s_ffail = 1;
                    bar_sync_n(2, 32 * nf);
                    if (s_ffail) break;
                    if (Ilast + 1 <= -1)
                        group_apply_right<T, MAXM>(V, PV, bw, j, min(d + 1, n - (c + j)), Ilast + 1, -1,
                                                   vR + j * MAXM, tbR[j * 4], F0);
                }
                bar_sync_n(2, 32 * nf);
                if (!s_ffail) {
                    // ---- ST1 and the half mark
                    group_copy<TS, T, false>(Wg, ldw, top, n, c, 0, KD - 1, col, [&](int X, int& lo, int& hi) {
                        lo = max(0, X - d) - vt;
                        hi = -1;
                    }, F0);
                    bar_sync_n(2, 32 * nf);
                    if (tid == 32 * F0 && !stall) st_release(my, base + 2 * s + 1);
                    // ---- W2: group g-1 did the upper part of step s+1 (or finished)
                    if (tid == 32 * F0)
                        s_ok2 = (g == 0) ? 1 : (int)wait_at_least(pred, base + (s + 1 < Sp ? 2 * (s + 1) + 1 : 2 * Sp),
                                                                  L.hdr, L.timeout_ns);
                    bar_sync_n(2, 32 * nf);
                    if (s_ok2) {
                        // ---- LD2: the tail columns and the next carried block
                        group_copy<TS, T, true>(Wg, ldw, top, n, c, bw - (g > 0 ? K : 0), bw + KD - 1, col,
                                                [&](int X, int& lo, int& hi) { lo = max(0, X - d - bw); hi = KD - 1; },
                                                F0);
                        cp_async_wait_all();
                        bar_sync_n(2, 32 * nf);
                        // ---- the left reflectors on the columns X >= K+d
                        for (int j = 0; j < ka; ++j) {
                            const int m = min(d + 1, n - (c + j));
                            const int jmax = min(n - 1 - c, j + m - 1 + bw);
                            if (jmax < KD) continue;
                            if (lead && !warp_wait_flag(&s_lflag, fb + j + 1, L.hdr, L.timeout_ns) && lane == 0)
                                s_ffail = 1;
                            bar_sync_n(2, 32 * nf);
                            if (s_ffail) break;
                            group_apply_left<T, MAXM>(col, j, m, KD, jmax, vL + j * MAXM, tbL[j * 4], F0);
                        }
                    }
                }
            }
            __syncthreads();
            if (!s_ok2 || s_nfail || s_ffail) { ok = false; break; }
            // ---- ST2 (the carried block too on the last step)
            group_copy<TS, T, false>(Wg, ldw, top, n, c, 0, KD - 1, col, [&](int X, int& lo, int& hi) {
                lo = 0;
                hi = min(K - 1, X) + d;
            });
            group_copy<TS, T, false>(Wg, ldw, top, n, c, KD, s == S - 1 ? bw + KD - 1 : bw - 1, col,
                                     [&](int X, int& lo, int& hi) { lo = max(0, X - d - bw); hi = KD - 1; });
            __syncthreads();
            if (tid == 0) {
                int w_ok = 1;
                if (s == S - 1 && g > 0) w_ok = (int)wait_at_least(pred, base + 2 * Sp, L.hdr, L.timeout_ns);
                if (w_ok && !stall) st_release(my, base + 2 * (s + 1));
                s_ok = w_ok;
            }
            __syncthreads();
            if (!s_ok) { ok = false; break; }
        }
        if (!ok) break;
    }
}

}  // namespace bb
