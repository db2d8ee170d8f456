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
// reflector, applied to the rows above c; store those rows and publish
// "upper part of step s done"; wait until group g-1 did the upper part of step
// s+1 (it writes the tail columns); load the tail and the next carried block;
// phase L: per member the right reflector on the rows at or below c, then the
// left reflector; store; publish "step s complete".  Members work step by
// step, not sweep by sweep: member j+1's left reflector at step s runs before
// member j's right reflector at step s+1; the two transform disjoint
// generating vectors and a common block that each transforms whole, so they
// commute (equal in exact arithmetic).  Across groups the order of every
// conflicting pair is the sequential one.  3K + d <= bw keeps group g-2's step
// s+2 out of group g's window.  The host model in tests/test_group_protocol.py
// checks all of this element by element.
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
    // vR[kmax][maxm], tbR[kmax][4], vL[2][maxm+1], tbL[2][4], xb[maxm+1], ts[64], 16-byte rounding
    return ((kmax * maxm + kmax * 4 + 2 * (maxm + 1) + 8 + (maxm + 1) + 64) + 3) & ~3;
}
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

// Copy window columns [x_lo, x_hi] between the working band and shared
// memory (LOAD: band -> shared with cp.async; else shared -> band), one warp
// per column, rows rows(X) = [lo, hi] clipped to the matrix.  Element
// (c + I, c + X) of the band is at Wg[(c + X) * ldw + top - X + I].
template <typename TS, typename T, bool LOAD, typename Rows>
__device__ __forceinline__ void group_copy(TS* __restrict__ Wg, int ldw, int top, int n, int c,
                                           int x_lo, int x_hi, const GroupCols<T>& col, Rows rows)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
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

template <typename TS, typename T, int MAXM>
__global__ void __launch_bounds__(384, 2) group_kernel(Launch L)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int KMAX = L.gK;
    T* const vR = (T*)smem_raw;                 // KMAX x MAXM right reflector vectors
    T* const tbR = vR + KMAX * MAXM;            // KMAX x {tau, beta, vs, -}
    T* const vL = tbR + KMAX * 4;               // left reflector vectors (two, alternating)
    T* const tbL = vL + 2 * (MAXM + 1);         // their {tau, beta, vs, -}
    T* const xb = tbL + 8;                      // staged reflector input
    T* const ts = xb + MAXM + 1;                // reflector scratch (64)
    T* const V = (T*)smem_raw + group_small_elems(KMAX, MAXM);
    __shared__ int s_task[2];
    __shared__ int s_ok;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
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

            // ---- phase U: right reflectors, rows above c
            for (int j = 0; j < ka; ++j) {
                const int m = min(d + 1, n - (c + j));
                const int Ij = j - vt;
                T* vj = vR + j * MAXM;
                T* tj = tbR + j * 4;
                if (warp == 0) {
                    for (int t = lane; t < m; t += 32) xb[t] = V[(j + t) * PV + Ij + bw];
                    __syncwarp();
                    fast_reflector<T, MAXM>(m, xb, vj, tj);
                    __syncwarp();
                    for (int t = lane; t < m; t += 32) V[(j + t) * PV + Ij + bw] = t == 0 ? tj[1] : (T)0;
                }
                __syncthreads();
                if (Ij + 1 <= -1) group_apply_right<T, MAXM>(V, PV, bw, j, m, Ij + 1, -1, vj, tj[0]);
                __syncthreads();
            }
            // ---- ST1 and the half mark
            group_copy<TS, T, false>(Wg, ldw, top, n, c, 0, KD - 1, col, [&](int X, int& lo, int& hi) {
                lo = max(0, X - d) - vt;
                hi = -1;
            });
            __syncthreads();
            if (tid == 0 && !stall) st_release(my, base + 2 * s + 1);

            // ---- W2: group g-1 did the upper part of step s+1 (or finished)
            if (tid == 0)
                s_ok = (g == 0) ? 1 : (int)wait_at_least(pred, base + (s + 1 < Sp ? 2 * (s + 1) + 1 : 2 * Sp),
                                                         L.hdr, L.timeout_ns);
            __syncthreads();
            if (!s_ok) { ok = false; break; }
            // ---- LD2: the tail columns and the next carried block
            group_copy<TS, T, true>(Wg, ldw, top, n, c, bw - (g > 0 ? K : 0), bw + KD - 1, col,
                                    [&](int X, int& lo, int& hi) { lo = max(0, X - d - bw); hi = KD - 1; });
            cp_async_wait_all();
            __syncthreads();

            // ---- phase L: per member, right reflector on rows >= c, left reflector
            for (int j = 0; j < ka; ++j) {
                const int m = min(d + 1, n - (c + j));
                const int jmax = min(n - 1 - c, j + m - 1 + bw);
                const T* vj = vR + j * MAXM;
                group_apply_right<T, MAXM>(V, PV, bw, j, m, 0, j + m - 1, vj, tbR[j * 4]);
                __syncthreads();
                if (warp == 0) {
                    T* x = V + j * PV + bw + j;          // column j, rows j .. j+m-1
                    fast_reflector<T, MAXM>(m, x, vL, tbL);
                    __syncwarp();
                    for (int t = lane; t < m; t += 32) x[t] = t == 0 ? tbL[1] : (T)0;
                }
                __syncthreads();
                if (j + 1 <= jmax) group_apply_left<T, MAXM>(col, j, m, j + 1, jmax, vL, tbL[0]);
                __syncthreads();
            }
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
