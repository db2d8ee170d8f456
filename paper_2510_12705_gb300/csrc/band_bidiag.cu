// Band -> bidiagonal reduction by Householder bulge chasing on sm_103a
// (arXiv 2510.12705, Section III: Algorithm 1 schedule, Algorithm 2 row-bulge).
//
// One persistent launch per bandwidth-reduction stage runs that stage for
// every problem of the call.  CTAs claim tasks (problem, sweep) from a global
// counter, round-robin over the problems; a task runs the row-bulges of one
// sweep.  Consecutive sweeps of a stage are separated by the dependency
// distance of Section III-A: sweep R may start row-bulge s once sweep R-1 has
// finished row-bulge s + L - 2, and the part of its left panel that row-bulge
// s + L - 1 of sweep R-1 also touches waits for that row-bulge's right half
// (a half-step progress mark), with L = 2 when the post-stage bandwidth is at
// least 2 and L = 3 otherwise.  Stage i+1 starts when
// the launch of stage i has ended (stream order, the paper's stage barrier).
// Because tasks are claimed in order and only wait on earlier tasks, the
// schedule cannot deadlock however many CTAs are resident.  Every wait is
// bounded.
//
// A row-bulge stages its right panel (rows r0..c+m-1 x columns c..c+m-1) and
// left panel (rows c..c+m-1 x columns c..jmax) in shared memory, builds each
// reflector with one warp (FP64 generation), applies it with two threads per
// row / column, and writes both panels back through L2.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/band_bidiag.h"
#include "bb_device.cuh"
#include "bb_group.cuh"
#include "bb_team.cuh"

using namespace bb;

static __device__ unsigned int g_bb_status;   // sticky device status (bits 1 << code)

// ------------------------------------------------------------------ kernels

template <typename T> __device__ __forceinline__ bool finite_val(T v)
{
    if constexpr (sizeof(T) >= 4) return isfinite(v);
    else return isfinite(to_float(v));
}

template <typename T>
__global__ void pack_kernel(Launch L)
{
    const int lane = threadIdx.x & 31;
    const int64_t wg = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t gc = wg; gc < L.total_cols; gc += nw) {
        const int q = find_problem_by_col(L, gc);
        const Desc& D = desc_of(L, q);
        const int j = (int)(gc - D.col_prefix);
        T* wcol = (T*)L.wbase + D.w_off + (int64_t)j * D.ldw;
        const T* bcol = (const T*)D.band + (int64_t)j * D.ldab;
        bool bad = false;
        for (int off = lane; off < D.ldw; off += 32) {
            const int i = j - D.top + off;   // matrix row of this slot
            const int k = j - i;             // superdiagonal offset
            T v = (T)0;
            if (i >= 0 && k >= 0 && k <= D.b) {
                v = bcol[D.b_in - k];
                bad |= !finite_val(v);
            }
            wcol[off] = v;
        }
        if (__any_sync(FULL, bad) && lane == 0) atomicOr(&L.hdr->err, 1 << 5);
    }
}

template <typename T>
__global__ void extract_kernel(Launch L)
{
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nt = (int64_t)gridDim.x * blockDim.x;
    for (int64_t gc = t0; gc < L.total_cols; gc += nt) {
        const int q = find_problem_by_col(L, gc);
        const Desc& D = desc_of(L, q);
        const int i = (int)(gc - D.col_prefix);
        const T* W = (const T*)L.wbase + D.w_off;
        ((T*)D.d)[i] = W[(int64_t)D.top + (int64_t)i * D.ldw];
        if (i + 1 < D.n) ((T*)D.e)[i] = W[(int64_t)(D.top - 1) + (int64_t)(i + 1) * D.ldw];
    }
    if (t0 == 0) {
        const int err = L.hdr->err;
        if (err) atomicOr(&g_bb_status, (unsigned)err);
    }
}

// ------------------------------------------------------------- row-bulge
// Shared-memory panels (odd pitch MAXM: conflict-free, compile-time offsets):
//   RP  right panel, row-major: panel row ri (matrix row r0+ri), column k at
//       RP[ri*MAXM + k]
//   LP  left panel, column-major: column jj (matrix column c+jj), row k
//       (matrix row c+k) at LP[jj*MAXM + k]
// Warp 0 computes each reflector; the other warps ("workers") own the rows and
// columns, two threads per row / column (thread p in {0,1} of a pair holds
// entries [p*H, p*H+H); one shuffle combines their partial dot products).
template <int MAXM> struct Split { static constexpr int H = (MAXM + 1) / 2; };


// e / div for 0 <= e < 2^22, div >= 1, via an FP32 reciprocal plus correction
__device__ __forceinline__ int fast_div(int e, int div, float inv)
{
    int q = (int)((float)e * inv);
    int r = e - q * div;
    if (r < 0) --q;
    else if (r >= div) ++q;
    return q;
}

// left-panel columns jj in [lo, hi) back to the working band (exact rows):
// element e of the block goes to row e mod m of column lo + e / m, so
// consecutive threads write consecutive rows of a column
template <typename TS, typename T, int MAXM>
__device__ __forceinline__ void left_store(const T* LP, TS* __restrict__ W, int ldw, int top, int c,
                                           int m, int lo, int hi)
{
    const float invM = 1.0f / (float)m;
    for (int e = threadIdx.x; e < (hi - lo) * m; e += blockDim.x) {
        const int q = fast_div(e, m, invM), k = e - q * m, jj = lo + q;
        panel_to_band<TS, T>(W + (int64_t)(c + jj) * ldw + (top - jj + k), LP[jj * MAXM + k]);
    }
}

// One row-bulge (Algorithm 2) of sweep R, stage (bw, d), on the CTA.
//
// A: every thread issues its share of the panel loads (right panel rows
//    r0..c+m-1 x columns c..c+m-1 -> RP; left panel columns c+m.. before the
//    tail, rows c..c+m-1 -> LP), U loads in flight per batch.
// B: warp 0 scales row r0 and builds the right reflector; meanwhile, as soon
//    as the scaled row is published (named barrier), the workers form the
//    dot products of the other rows with it: row.v = row_0 + vs * sum_k>0
//    row_k t_k.  C: workers update the rows; rows above c go back to the
//    working band, rows c..c+m-1 (shared with the left panel) into LP.
// D/E: the same for the left reflector (column c) and the left panel's
//    columns, which are then stored one warp per column.
// The left panel's tail columns (offset >= tail_start) are the only part the
// previous sweep's next row-bulge also writes, and only through its right
// reflector: they are loaded after that row-bulge has published its right half
// (tail_prog >= tail_target) and updated straight from registers.  This
// row-bulge publishes its own right half (half_prog = half_value) after C.
// Returns false when a wait gave up.
template <typename TS, typename T, int MAXM>
__device__ __forceinline__ bool row_bulge(const Launch& L, const Desc& D, TS* __restrict__ W, int bw, int d, int R,
                                          int s, T* RP, T* LP, T* wbuf, T* tsR, T* tsL, T* vR, T* vL,
                                          T* tb, int* s_flag, const int* tail_prog, int tail_target,
                                          int tail_start, Header* hdr, unsigned long long timeout_ns,
                                          int* half_prog, int half_value, bool carried, bool carry_out)
{
    constexpr int H = Split<MAXM>::H;
    const int n = D.n, ldw = D.ldw, top = D.top;
    const int c = R + (bw - d) + s * bw;
    const int m = min(d + 1, n - c);
    const int r0 = (s == 0) ? R : c - bw;
    const int nr = c + m - r0;                 // panel rows r0 .. c+m-1 (panel row 0 = r0)
    const int jmax = min(n - 1, c + m - 1 + bw);
    const int ncols = jmax - c;                // columns c+1 .. jmax (offset jj = 1..ncols)
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int wt = tid - 32, nwt = nt - 32;    // worker index / count (warps 1..)
    const int p = tid & 1, k0 = p * H;
    const int pre_hi = min(tail_start, ncols + 1);   // left-panel columns loaded up front

    // ---- A: loads (with `carried`, panel rows 0..d are already in RP: the
    //      previous row-bulge's m = d + 1 rows, also where this one's m is
    //      smaller at the end of the matrix).  Every element is one cp.async,
    //      so all of a thread's copies are in flight at once.
    {
        const int ri_lo = carried ? d + 1 : 0, nrl = nr - ri_lo;
        const int totR = nrl * m, totL = (pre_hi - m) * m, tot = totR + totL;
        const float invR = 1.0f / (float)max(nrl, 1), invM = 1.0f / (float)m;
        for (int e = tid; e < tot; e += nt) {
            if (e < totR) {
                const int k = fast_div(e, nrl, invR), ri = ri_lo + e - k * nrl;
                band_to_panel<TS, T>(RP + ri * MAXM + k, W + (int64_t)(c + k) * ldw + (r0 + ri - c - k + top));
            } else {
                const int f = e - totR;
                const int q = fast_div(f, m, invM), k = f - q * m, jj = m + q;
                band_to_panel<TS, T>(LP + jj * MAXM + k, W + (int64_t)(c + jj) * ldw + (top - jj + k));
            }
        }
        cp_async_wait_all();
    }
    __syncthreads();

    // ---- B: right reflector (warp 0; already built when `carried`) || row dot
    //      products (workers)
    if (warp == 0) {
        if (!carried) {
            const ReflScale sc = reflector_scale<T>(m, RP, tsR);
            bar_arrive(1, nt);
            reflector_finish<T>(m, sc, vR, tb);
            if (L.refl) {
                __syncwarp();
                warp_store_reflector<T, MAXM>(L, n, bw, d, R, s, 0, m, vR, tb[0]);
            }
        }
    } else {
        if (!carried) bar_sync_n(1, nt);
        for (int ri = 1 + (wt >> 1); ri - (wt >> 1) < nr; ri += nwt >> 1) {
            T w = (T)0;
            if (ri < nr) {
                const T* row = RP + ri * MAXM + k0;
#pragma unroll
                for (int i = 0; i < H; ++i)
                    if (k0 + i >= 1 && k0 + i < m) w = fma(row[i], tsR[k0 + i], w);
            }
            w += __shfl_xor_sync(FULL, w, 1);
            if (ri < nr && p == 0) wbuf[ri] = w;
        }
    }
    __syncthreads();

    // ---- C: row updates.  C1: the panel rows c..c+m-1, which become the left
    //      panel's first columns (and column c, the left reflector's input), by
    //      the first worker pairs; their warps then signal warp 0 (named
    //      barrier 2), which starts the left reflector at once.  C2: the rows
    //      r0..c-1 back to the working band by all workers; after a workers-only
    //      barrier (3) one lane of the last warp publishes the right half.
    const int np = nwt >> 1, pi = wt >> 1;     // worker pairs, this thread's pair
    const int ri_c = c - r0;                   // first panel row at or below c
    const int c1_warps = (2 * min(m, np) + 31) >> 5;
    T* tbL = tb + 4;
    // The left panel's tail columns (offsets pre_hi..ncols) are loaded during D
    // by the last warp, after the previous sweep's progress word says that its
    // next row-bulge has done the part that touches them; with three or more
    // warps that warp takes no part in D's dot products (named barrier 1 then
    // counts the other threads).
    const int nw = nt >> 5;
    const bool has_tail = pre_hi <= ncols;
    const bool tail_apart = has_tail && nw >= 3;
    const int d_count = tail_apart ? nt - 32 : nt;
    const int np_d = tail_apart ? np - 16 : np;
    if (warp == 0) {
        bar_sync_n(2, 32 * (1 + c1_warps));
        // ---- D: left reflector (warp 0) || column dot products (workers)
        const ReflScale sc = reflector_scale<T>(m, LP, tsL);
        bar_arrive(1, d_count);
        reflector_finish<T>(m, sc, vL, tbL);
        if (L.refl) {
            __syncwarp();
            warp_store_reflector<T, MAXM>(L, n, bw, d, R, s, 1, m, vL, tbL[0]);
        }
    } else {
        const T tau = tb[0], vs = tb[2];
        for (int ri = ri_c + pi; ri < nr; ri += np) {             // C1 -> LP
            const T* row = RP + ri * MAXM + k0;
            const T u = tau * fma(vs, wbuf[ri], RP[ri * MAXM]);
#pragma unroll
            for (int i = 0; i < H; ++i)
                if (k0 + i < m) LP[(k0 + i) * MAXM + (ri - ri_c)] = fma(-u, vR[k0 + i], row[i]);
        }
        if (warp <= c1_warps) bar_arrive(2, 32 * (1 + c1_warps));
        for (int ri = pi; ri < ri_c; ri += np) {                   // C2 -> band
            const int r = r0 + ri;
            TS* dst = W + (int64_t)(c + k0) * ldw + (r - c - k0 + top);   // (r, c+k0)
            if (ri == 0) {            // the bulge row: (beta, 0, ..., 0)
#pragma unroll
                for (int i = 0; i < H; ++i)
                    if (k0 + i < m) panel_to_band<TS, T>(dst + (int64_t)i * (ldw - 1), k0 + i == 0 ? tb[1] : (T)0);
            } else {
                const T* row = RP + ri * MAXM + k0;
                const T u = tau * fma(vs, wbuf[ri], RP[ri * MAXM]);
#pragma unroll
                for (int i = 0; i < H; ++i)
                    if (k0 + i < m) panel_to_band<TS, T>(dst + (int64_t)i * (ldw - 1), fma(-u, vR[k0 + i], row[i]));
            }
        }
        bar_sync_n(3, nt - 32);
        // the right reflector's results outside the left panel are in the
        // working band: the next sweep's previous row-bulge may now finish its
        // tail.  The release waits until the stores are performed, so it is
        // issued from the last warp, not the reflector warp.
        if (tid == nt - 32 && half_prog) st_release(half_prog, half_value);
        if (has_tail && warp == nw - 1) {
            // tail: wait (lane 0; the shuffle and __syncwarp order the other
            // lanes' copies after its acquire), then copy the columns into LP
            int t_ok = 1;
            if (lane == 0 && tail_prog) t_ok = (int)wait_at_least(tail_prog, tail_target, hdr, timeout_ns);
            t_ok = __shfl_sync(FULL, t_ok, 0);
            __syncwarp();
            if (t_ok) {
                const float invM = 1.0f / (float)m;
                for (int e = lane; e < (ncols + 1 - pre_hi) * m; e += 32) {
                    const int q = fast_div(e, m, invM), k = e - q * m, jj = pre_hi + q;
                    band_to_panel<TS, T>(LP + jj * MAXM + k, W + (int64_t)(c + jj) * ldw + (top - jj + k));
                }
                cp_async_wait_all();
            }
            if (lane == 0) *s_flag = t_ok;
        }
        if (!(tail_apart && warp == nw - 1)) {
            bar_sync_n(1, d_count);
            for (int jj = 1 + pi; jj - pi < pre_hi; jj += np_d) {
                T w = (T)0;
                if (jj < pre_hi) {
                    const T* col = LP + jj * MAXM + k0;
#pragma unroll
                    for (int i = 0; i < H; ++i)
                        if (k0 + i >= 1 && k0 + i < m) w = fma(col[i], tsL[k0 + i], w);
                }
                w += __shfl_xor_sync(FULL, w, 1);
                if (jj < pre_hi && p == 0) wbuf[jj] = w;
            }
        }
    }
    __syncthreads();
    if (has_tail && !*s_flag) return false;

    // ---- E: column updates in LP (the tail columns' dot products here too),
    //      then stores.  Each pair reads its column into registers first and
    //      shares the row-c entry by shuffle, so no lane overwrites an entry its
    //      partner still has to read.
    const T tauL = tbL[0], vsL = tbL[2];
    if (warp == 0) {
        for (int k = lane; k < m; k += 32) LP[k] = k == 0 ? tbL[1] : (T)0;
    } else {
        for (int jj = 1 + pi; jj - pi <= ncols; jj += np) {
            const bool act = jj <= ncols;
            T* col = LP + jj * MAXM + k0;
            T a[H];
            T w = (T)0;
#pragma unroll
            for (int i = 0; i < H; ++i) {
                a[i] = (act && k0 + i < m) ? col[i] : (T)0;
                if (jj >= pre_hi && k0 + i >= 1 && k0 + i < m) w = fma(a[i], tsL[k0 + i], w);
            }
            w += __shfl_xor_sync(FULL, w, 1);
            const T a0 = __shfl_sync(FULL, a[0], lane & ~1);
            const T dot = (act && jj < pre_hi) ? wbuf[jj] : w;
            const T u = tauL * fma(vsL, dot, a0);
#pragma unroll
            for (int i = 0; i < H; ++i)
                if (act && k0 + i < m) col[i] = fma(-u, vL[k0 + i], a[i]);
        }
    }
    __syncthreads();
    // With `carry_out`, left-panel columns bw .. bw+m'-1 are the next row-bulge's
    // right panel rows 0..m-1 (its bulge row is row c): they stay in RP (free
    // since C) instead of a round trip through L2; the next row-bulge writes
    // them back in its phase C, before any other sweep may read them.
    const int keep_lo = carry_out ? min(bw, ncols + 1) : ncols + 1;
    left_store<TS, T, MAXM>(LP, W, ldw, top, c, m, 0, keep_lo);
    for (int idx = tid; idx < (ncols + 1 - keep_lo) * m; idx += nt) {
        const int jj = keep_lo + idx / m, k = idx - (jj - keep_lo) * m;
        RP[k * MAXM + (jj - bw)] = LP[jj * MAXM + k];
    }
    return true;
}

// One bandwidth-reduction stage (Algorithm 1, all sweeps) of every problem:
// a persistent launch in which CTAs claim sweeps in order.  Sweep R may start
// row-bulge s once sweep R-1 has finished row-bulge s (s+1 when the stage ends
// at bandwidth 1), and its left panel's tail waits for the right half of
// row-bulge s+1 (s+2) of sweep R-1: the Section III-A separation of 2 (3)
// row-bulges, with the overlap the footprints allow.
template <typename TS, typename T, int MAXM>
__global__ void __launch_bounds__(512) bulge_kernel(Launch L)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* RP = (T*)smem_raw;                                  // right panel, L.rp_rows rows
    T* LP = RP + (size_t)MAXM * L.rp_rows;                 // left panel, L.lp_cols columns
    T* wbuf = LP + (size_t)MAXM * L.lp_cols;               // per row / column dot products
    __shared__ T vR[64], vL[64], tsR[64], tsL[64], tb[8];
    __shared__ int s_task[4];
    __shared__ int s_ok;         // result of the per-step wait
    __shared__ int s_tail_ok;    // result of the tail wait inside a row-bulge
    const int tid = threadIdx.x, nt = blockDim.x;
    const int stage = L.stage;

    for (;;) {
        // Tasks go round-robin over the problems (task t: problem t mod count,
        // sweep t div count), so every problem's sweep chain advances at once;
        // a task only waits on a smaller task index, so claiming in order
        // cannot deadlock.
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
        const int R = s_task[1];
        const Desc& D = desc_of(L, q);
        __syncthreads();   // s_task may be rewritten on the next claim
        if (stage >= D.nstages || R >= D.n - 1) continue;

        const int n = D.n;
        const int bw = stage_bw(D.b, L.tw, stage);
        const int d = stage_d(bw, L.tw);
        if (L.gK > 0 && group_members(bw, d, L.gK) >= 1) continue;   // the group kernel's
        if (L.team > 0 && bw - d == 1) continue;                      // the team kernel's
        const bool split = (bw - d) >= 2;
        const int base = stage * PROG_STAGE;
        int* prog = L.prog + D.prog_off;
        const int ps = L.prog_stride;
        const int ns = sweep_steps(n, bw, d, R);
        const int nsp = (R > 0) ? sweep_steps(n, bw, d, R - 1) : 0;
        TS* W = (TS*)L.wbase + D.w_off;
        const bool stall = (L.flags & BB_FLAG_INJECT_STALL) && stage == 0 && R == 0;

        // Waits on sweep R-1 (progress values relative to the stage base):
        //   split stage (bw - d >= 2): row-bulge s starts once row-bulge s of
        //     R-1 is complete; the left panel's tail (offsets >= bw-1) once the
        //     right half of row-bulge s+1 of R-1 is done (all of it when
        //     bw - d == 2: there the left half of row-bulge s+1 of sweep R-2
        //     reaches the tail rows too).
        //   final stage (bw - d == 1): row-bulge s starts once row-bulge s+1 of
        //     R-1 is complete; the tail is the last left-panel column (offset
        //     d + bw), which only the right half of row-bulge s+2 of R-1 shares.
        //   last row-bulge of the sweep: its completion is published only once
        //     sweep R-1 is complete, so a completed sweep vouches for the whole
        //     chain before it (a sweep can be one row-bulge shorter than R-1).
        // The protocol is checked against every row-bulge's footprint on the
        // host (serialisable: same result as the sequential sweep order).
        const int pre_ahead = split ? 1 : 2;
        const int tail_ahead = split ? 1 : 2;
        const int tail_half = split ? (bw - d >= 3 ? 1 : 2) : 1;
        const int tail_start = split ? bw - 1 : d + bw;
        // From row-bulge 1 on, the bulge row and the rows below it up to c+m-1
        // come from this CTA's previous row-bulge (kept in RP): warp 0 builds
        // the right reflector from them while another thread waits on sweep R-1.
        bool ok = true;
        bool carried = false;
        for (int s = 0; s < ns; ++s) {
            if (carried && tid < 32) {
                const int cs = R + (bw - d) + s * bw;
                warp_reflector<T>(min(d + 1, n - cs), RP, tsR, vR, tb);
                if (L.refl) {
                    __syncwarp();
                    warp_store_reflector<T, MAXM>(L, n, bw, d, R, s, 0, min(d + 1, n - cs), vR, tb[0]);
                }
            }
            if (tid == (carried ? 32 : 0)) {
                bool w_ok = true;
                if (R > 0)
                    w_ok = wait_at_least(&prog[(R - 1) * ps], base + 2 * min(s + pre_ahead, nsp),
                                         L.hdr, L.timeout_ns);
                s_ok = w_ok;
            }
            __syncthreads();
            if (!s_ok) { ok = false; break; }
            const bool carry_out = s + 1 < ns;
            const bool step_ok = row_bulge<TS, T, MAXM>(
                L, D, W, bw, d, R, s, RP, LP, wbuf, tsR, tsL, vR, vL, tb, &s_tail_ok,
                R > 0 ? &prog[(R - 1) * ps] : nullptr,
                base + (s + tail_ahead < nsp ? 2 * (s + tail_ahead) + tail_half : 2 * nsp),
                tail_start, L.hdr, L.timeout_ns,
                stall ? nullptr : &prog[R * ps], base + 2 * s + 1, carried, carry_out);
            carried = carry_out;
            __syncthreads();
            if (!step_ok) { ok = false; break; }
            if (s == ns - 1) {
                if (tid == 0) {
                    bool w_ok = true;
                    if (R > 0)
                        w_ok = wait_at_least(&prog[(R - 1) * ps], base + 2 * nsp, L.hdr, L.timeout_ns);
                    if (w_ok && !stall) st_release(&prog[R * ps], base + 2 * s + 2);   // cumulative
                    s_ok = w_ok;
                }
                __syncthreads();
                if (!s_ok) { ok = false; break; }
            } else if (tid == nt - 32 && !stall) {
                // completion of row-bulge s: issued by one lane of the last warp
                // while warp 0 builds the next right reflector and thread 32
                // waits on sweep R-1, so the release's wait for the stores is
                // off their path (the barrier before the next loads orders it)
                st_release(&prog[R * ps], base + 2 * s + 2);
            }
        }
        if (!ok) break;
        if (tid == 0 && !stall && ns == 0) st_release(&prog[R * ps], base);
    }
}

// ---------------------------------------------------- back-transformation
// The orthogonal factors of B = Q^T A P from the reflectors the reduction
// stored (Section VII names the back-transformation of the stored reflectors
// as the step that turns the method into a singular-vector solver).  In the
// sequential order of the reduction (stage, sweep, row-bulge), Q = H_L1 H_L2 ...
// and P = H_R1 H_R2 ..., each H = I - tau v v^T acting on the m = min(d+1, n-c)
// columns c .. c+m-1 of its row-bulge (c = R + bw' + s bw).  X <- X H touches
// every row of X independently, so each thread owns one row of X, starts from
// the identity and applies every reflector of its side in that order.  The
// GPU's own order of the reflectors differs from the sequential one only in
// pairs that act on opposite sides (Section III-A schedule), which the product
// of one side does not see.
template <typename T>
__global__ void identity_kernel(T* __restrict__ X, int64_t ldx, int n)
{
    const int64_t total = (int64_t)n * n;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(t / n), i = (int)(t % n);
        X[i + (int64_t)j * ldx] = (T)(i == j ? 1 : 0);
    }
}

// The two sides are independent (blockIdx.y = 1: the left reflectors into Q,
// 0: the right ones into P) and run in one launch; one warp per CTA spreads
// the rows over every SM, since each row's FP64 work is a long dependent
// chain.  The dot product keeps four partial sums to shorten that chain.
template <typename T, int MAXM>
__global__ void __launch_bounds__(32) backtransform_kernel(int n, int b, int tw, const T* __restrict__ refl,
                                                           T* __restrict__ Xq, int64_t ldq, T* __restrict__ Xp,
                                                           int64_t ldp)
{
    const int side = blockIdx.y;
    T* const X = side ? Xq : Xp;
    const int64_t ldx = side ? ldq : ldp;
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    T* row = X + r;
    int64_t k = 0;
    for (int bw = b; bw > 1;) {
        const int d = min(tw, bw - 1);
        for (int R = 0; R < n - 1; ++R) {
            const int ns = sweep_steps(n, bw, d, R);
            for (int s = 0; s < ns; ++s, ++k) {
                const int c = R + (bw - d) + s * bw;
                const int m = min(d + 1, n - c);
                const T* slot = refl + (2 * k + side) * (int64_t)refl_stride(MAXM);
                T x[MAXM], v[MAXM];
#pragma unroll
                for (int t = 0; t < MAXM; ++t) {
                    if (t < m) {
                        x[t] = row[(int64_t)(c + t) * ldx];
                        v[t] = __ldg(slot + t);
                    }
                }
                const T tau = __ldg(slot + MAXM);
                if (tau == (T)0) continue;
                T w0 = (T)0, w1 = (T)0, w2 = (T)0, w3 = (T)0;
#pragma unroll
                for (int t = 0; t < MAXM; t += 4) {
                    if (t < m) w0 = fma(x[t], v[t], w0);
                    if (t + 1 < MAXM && t + 1 < m) w1 = fma(x[t + 1], v[t + 1], w1);
                    if (t + 2 < MAXM && t + 2 < m) w2 = fma(x[t + 2], v[t + 2], w2);
                    if (t + 3 < MAXM && t + 3 < m) w3 = fma(x[t + 3], v[t + 3], w3);
                }
                const T f = tau * ((w0 + w1) + (w2 + w3));
#pragma unroll
                for (int t = 0; t < MAXM; ++t)
                    if (t < m) row[(int64_t)(c + t) * ldx] = fma(-f, v[t], x[t]);
            }
        }
        bw -= d;
    }
}

// ------------------------------------------------------------------- host

namespace {

constexpr size_t kAlign = 256;
inline size_t align_up(size_t x, size_t a = kAlign) { return (x + a - 1) / a * a; }

int clamp_b(int64_t n, int64_t b) { return (int)std::min<int64_t>(b, std::max<int64_t>(n - 1, 0)); }

bool dtype_ok(int dtype) { return dtype == BB_F32 || dtype == BB_F64 || dtype == BB_F16 || dtype == BB_BF16; }
int storage_size(int dtype) { return dtype == BB_F64 ? 8 : dtype == BB_F32 ? 4 : 2; }

int num_stages(int b, int tw)
{
    int st = 0;
    for (int bw = b; bw > 1; bw -= std::min(tw, bw - 1)) ++st;
    return st;
}

int maxm_for(int tw)
{
    if (tw <= 4) return 5;
    if (tw <= 8) return 9;
    if (tw <= 16) return 17;
    return 33;
}

// sweeps per CTA of the group kernel when the tuning leaves it open
constexpr int kDefaultGroup = 24;
// sweeps per CTA of the team kernel (last stage) when the tuning leaves it
// open: 0, the per-sweep kernel runs the last stage unless a tuning asks for
// the team kernel (it is slower than the per-sweep kernel as it stands)
constexpr int kDefaultTeams = 0;

struct Resolved {
    int dtype, tw, tpb, sif, flags, group, teams;
    unsigned long long timeout_ns;
    cudaEvent_t ev_start, ev_stop;
    void** ev_launch;
    int ev_count;
    int* launch_log;
};

bool resolve_tuning(int64_t n, int64_t b, int dtype, const bb_tuning* t, Resolved* r)
{
    bb_tuning def;
    bb_default_tuning(n, b, dtype, &def);
    r->dtype = dtype;
    r->tw = (t && t->tw > 0) ? t->tw : def.tw;
    r->tpb = (t && t->tpb > 0) ? t->tpb : def.tpb;
    r->sif = (t && t->sweeps_in_flight > 0) ? t->sweeps_in_flight : 0;
    r->flags = t ? t->flags : 0;
    r->group = (t && t->group != 0) ? (t->group < 0 ? 0 : t->group) : kDefaultGroup;
    r->teams = (t && t->teams != 0) ? (t->teams < 0 ? 0 : t->teams) : kDefaultTeams;
    const double to = (t && t->timeout_s > 0) ? t->timeout_s : def.timeout_s;
    r->timeout_ns = (unsigned long long)(to * 1e9);
    r->ev_start = t ? (cudaEvent_t)t->ev_start : nullptr;
    r->ev_stop = t ? (cudaEvent_t)t->ev_stop : nullptr;
    r->ev_launch = t ? t->ev_launch : nullptr;
    r->ev_count = t ? t->ev_count : 0;
    r->launch_log = t ? t->launch_log : nullptr;
    if (r->tw < 1 || r->tw > 32) return false;
    if (r->tpb != 0 && (r->tpb < 64 || r->tpb > 512 || r->tpb % 32 != 0)) return false;
    if (t && (t->group < -1 || t->teams < -1)) return false;
    if (r->group > 64) r->group = 64;
    if (r->teams > 4) r->teams = 4;          // teams of kTeamWarps warps, plus a data warp

    return true;
}

struct LaunchPlan {
    Launch L;
    std::vector<Desc> descs;
    int esize = 8;
    int max_stages = 0;
    int max_b = 0;
    size_t off_hdr = 0, off_stage = 0, off_prog = 0, off_desc = 0, off_w = 0, bytes = 0;
    size_t smem = 0;
    size_t gsmem = 0;     // dynamic shared memory of the group kernel (0: not used)
    size_t tsmem = 0;     // dynamic shared memory of the team kernel (0: not used)
    Resolved tune;
};

// Dynamic shared memory of the group kernel with at most K sweeps per CTA:
// the largest window over the problems it takes on `stage` (every stage when
// stage < 0); 0 when it takes none.
size_t group_smem_bytes(const LaunchPlan& P, int K, int stage = -1)
{
    if (K < 1) return 0;
    const int tw = P.tune.tw, maxm = maxm_for(tw);
    const size_t es = P.tune.dtype == BB_F64 ? 8 : 4;
    int window = 0;
    for (const Desc& D : P.descs)
        for (int st = 0; st < D.nstages; ++st) {
            if (stage >= 0 && st != stage) continue;
            const int bw = D.b - st * tw, d = std::min(tw, bw - 1);
            const int k = group_members(bw, d, K);
            if (k >= 1) window = std::max(window, group_window_elems(bw, d, k));
        }
    if (window == 0) return 0;
    return es * (size_t)(group_small_elems(K, maxm) + window);
}

// Dynamic shared memory of the team kernel with W sweeps per CTA: the largest
// last-stage window over the problems (0 when no problem has a last stage).
size_t team_smem_bytes(const LaunchPlan& P, int W)
{
    if (W < 1) return 0;
    const int tw = P.tune.tw, maxm = maxm_for(tw);
    const size_t es = P.tune.dtype == BB_F64 ? 8 : 4;
    int elems = 0;
    for (const Desc& D : P.descs) {
        if (D.nstages < 1) continue;
        const int bw = D.b - (D.nstages - 1) * tw;     // the last stage ends at bandwidth 1
        elems = std::max(elems, team_smem_elems(bw, W, maxm));
    }
    return es * (size_t)elems;
}

// Lay out a launch for `count` problems (host-side planning, no CUDA calls).
int plan_launch(int count, const bb_problem* probs, int dtype, const bb_tuning* tuning,
                LaunchPlan* P)
{
    if (count < 1 || !probs || !dtype_ok(dtype)) return BB_ERR_ARG;
    int64_t nmax = 0, bmax = 0;
    for (int q = 0; q < count; ++q) {
        const bb_problem& p = probs[q];
        if (p.n < 1 || p.b < 0 || p.ldab < p.b + 1 || !p.band || !p.d_out) return BB_ERR_ARG;
        if (p.n > 1 && !p.e_out) return BB_ERR_ARG;
        if (p.n >= PROG_STAGE) return BB_ERR_UNSUPPORTED;
        nmax = std::max(nmax, p.n);
        bmax = std::max<int64_t>(bmax, clamp_b(p.n, p.b));
    }
    if (!resolve_tuning(nmax, bmax, dtype, tuning, &P->tune)) return BB_ERR_ARG;
    const int tw = P->tune.tw;
    P->esize = storage_size(dtype);
    P->descs.resize(count);
    int64_t sweep_prefix = 0, col_prefix = 0, welems = 0;
    int max_stages = 0, max_b = 0;
    for (int q = 0; q < count; ++q) {
        const bb_problem& p = probs[q];
        Desc& D = P->descs[q];
        std::memset(&D, 0, sizeof(D));
        D.n = (int)p.n;
        D.b = clamp_b(p.n, p.b);
        D.b_in = (int)p.b;
        D.nstages = num_stages(D.b, tw);
        D.top = D.b + tw;
        D.ldw = (int)align_up((size_t)(D.b + 2 * tw), 4) + 1;   // ldw - 1 multiple of 4
        D.w_off = welems;
        D.prog_off = col_prefix * (count == 1 ? 32 : 4);
        D.sweep_prefix = sweep_prefix;
        D.col_prefix = col_prefix;
        D.band = p.band;
        D.ldab = p.ldab;
        D.d = p.d_out;
        D.e = p.e_out;
        // + 16 elements: the 16-byte covers of the last columns may read past the band
        welems += (int64_t)align_up(((size_t)D.ldw * (size_t)D.n + 16) * P->esize) / P->esize;
        sweep_prefix += D.n - 1;
        col_prefix += D.n;
        max_stages = std::max(max_stages, D.nstages);
        max_b = std::max(max_b, D.b);
    }
    // progress words hold stage * PROG_STAGE + step marks in an int
    if (max_stages >= INT32_MAX / PROG_STAGE) return BB_ERR_UNSUPPORTED;
    P->max_stages = max_stages;
    P->max_b = max_b;
    size_t off = 0;
    P->off_hdr = off;   off = align_up(off + sizeof(Header));
    P->off_stage = off; off = align_up(off + sizeof(int) * (size_t)count);
    const int prog_stride = count == 1 ? 32 : 4;   // a 128-byte line per sweep when alone
    P->off_prog = off;  off = align_up(off + sizeof(int) * (size_t)col_prefix * prog_stride);
    P->off_desc = off;  off = align_up(off + (count > 1 ? sizeof(Desc) * (size_t)count : 0));
    P->off_w = off;     off = align_up(off + (size_t)welems * P->esize);
    P->bytes = off;

    Launch& L = P->L;
    std::memset(&L, 0, sizeof(L));
    L.count = count;
    L.descs = nullptr;
    L.single = P->descs[0];
    L.tw = tw;
    L.sweeps_per_stage = sweep_prefix;
    {
        int64_t nmax1 = 0;
        for (const Desc& D : P->descs) nmax1 = std::max<int64_t>(nmax1, D.n - 1);
        L.total_tasks = (int64_t)count * nmax1;   // tasks of one stage launch
    }
    L.total_cols = col_prefix;
    L.timeout_ns = P->tune.timeout_ns;
    L.flags = P->tune.flags;
    L.prog_stride = prog_stride;
    L.rp_rows = max_b + tw + 2;
    L.lp_cols = max_b + tw + 2;
    L.stage = 0;
    // panels hold the compute type: FP64 for the FP64 form, FP32 otherwise
    P->smem = (size_t)(dtype == BB_F64 ? 8 : 4) * ((size_t)maxm_for(tw) + 1) * (size_t)(L.rp_rows + L.lp_cols);
    if (L.total_tasks >= (int64_t)INT32_MAX) return BB_ERR_UNSUPPORTED;
    L.gK = P->tune.group;
    P->gsmem = group_smem_bytes(*P, L.gK);
    L.team = P->tune.teams;
    P->tsmem = team_smem_bytes(*P, L.team);
    return BB_OK;
}

void bind_workspace(LaunchPlan* P, void* ws)
{
    char* base = (char*)ws;
    P->L.hdr = (Header*)(base + P->off_hdr);
    P->L.stage_done = (int*)(base + P->off_stage);
    P->L.prog = (int*)(base + P->off_prog);
    P->L.wbase = base + P->off_w;
    if (P->L.count > 1) P->L.descs = (const Desc*)(base + P->off_desc);
}

// threads per bulge for a stage: two per panel row / column
int stage_tpb(int bw, int d, int user_tpb)
{
    if (user_tpb > 0) return user_tpb;
    int t = 2 * (bw + d + 1);        // two workers per panel row / column
    t = (t + 31) / 32 * 32 + 32;     // plus the reflector warp
    return std::max(96, std::min(512, t));
}

// threads of the group kernel for a stage: 16 panel rows / columns per warp
// and pass, one pass over the left reflector's columns
// (at most 384: the kernel is compiled for two CTAs of 384 threads per SM; at
// least 128: its three warp teams need four warps)
int group_tpb(int bw, int d, int user_tpb)
{
    if (user_tpb > 0) return std::max(128, std::min(user_tpb, 384));
    const int warps = (bw + d + 1 + 15) / 16;
    return std::max(128, std::min(384, 32 * warps));
}

template <typename K>
int set_smem(K kern, size_t bytes)
{
    if (bytes > 48 * 1024 &&
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) != cudaSuccess) {
        cudaGetLastError();   // not sticky: leave no error for the caller's next launch
        return BB_ERR_UNSUPPORTED;
    }
    return BB_OK;
}

// One launch per stage and kernel: the group kernel for the problems whose
// stage takes at least one sweep per group (3K + d <= bw), the team kernel for
// the problems on their last stage (it ends at bandwidth 1), the per-sweep
// kernel for the rest.  The three persistent kernels claim tasks in order from
// the header's counter, which is reset before every launch.
template <typename TS, typename T, int MAXM>
int launch_stages(const LaunchPlan& P, cudaStream_t st)
{
    auto kern = bulge_kernel<TS, T, MAXM>;
    auto gkern = group_kernel<TS, T, MAXM>;
    auto tkern = team_kernel<TS, T, MAXM>;
    int rc = set_smem(kern, P.smem);
    if (rc == BB_OK && P.gsmem) rc = set_smem(gkern, P.gsmem);
    if (rc == BB_OK && P.tsmem) rc = set_smem(tkern, P.tsmem);
    if (rc != BB_OK) return rc;
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (P.tune.ev_start && cudaEventRecord(P.tune.ev_start, st) != cudaSuccess) return BB_ERR_LAUNCH;
    Launch L = P.L;
    if (!P.gsmem) L.gK = 0;
    if (!P.tsmem) L.team = 0;
    bool first = true;
    int nlaunch = 0;
    int64_t refl_base = 0;    // row-bulges of the earlier stages (reflector store of one problem)
    for (int stage = 0; stage < P.max_stages; ++stage) {
        L.refl_base = refl_base;
        if (L.refl && stage < P.descs[0].nstages) {
            const Desc& D0 = P.descs[0];
            const int bw0 = D0.b - stage * L.tw, d0 = std::min(L.tw, bw0 - 1);
            refl_base += steps_before(D0.n, bw0, d0, D0.n);
        }
        // widest stage bandwidth over the problems of each kernel, and the
        // tasks (problems x groups) of the group and team kernels
        int bw_max = 0, d_max = 0, gbw_max = 0, gd_max = 0;
        int64_t gtasks = 0, ttasks = 0, gsteps = 0;
        bool any_sweep = false;
        for (const Desc& D : P.descs)
            if (stage < D.nstages) {
                const int bw = D.b - stage * L.tw, d = std::min(L.tw, bw - 1);
                const int k = L.gK ? group_members(bw, d, L.gK) : 0;
                if (k >= 1) {
                    gbw_max = std::max(gbw_max, bw);
                    gd_max = std::max(gd_max, d);
                    const int nact = D.n - 1 - (bw - d);
                    gtasks = std::max<int64_t>(gtasks, nact > 0 ? (nact + k - 1) / k : 0);
                    gsteps = std::max<int64_t>(gsteps, nact > 0 ? (D.n - 2 - (bw - d)) / bw + 1 : 0);
                } else if (L.team && bw - d == 1) {
                    const int nact = D.n - 2;
                    ttasks = std::max<int64_t>(ttasks, nact > 0 ? (nact + L.team - 1) / L.team : 0);
                } else {
                    any_sweep = true;
                    bw_max = std::max(bw_max, bw);
                    d_max = std::max(d_max, d);
                }
            }
        L.stage = stage;
        for (int which = 0; which < 3; ++which) {
            if (which == 0 ? gtasks == 0 : which == 1 ? ttasks == 0 : !any_sweep) continue;
            const int tpb = which == 0 ? group_tpb(gbw_max, gd_max, P.tune.tpb)
                          : which == 1 ? 32 * (L.team * kTeamWarps + 1)
                                       : stage_tpb(bw_max, d_max, P.tune.tpb);
            // the group kernel's window is sized for this stage, so later
            // (narrower) stages keep more CTAs per SM
            const size_t smem = which == 0 ? group_smem_bytes(P, L.gK, stage) : which == 1 ? P.tsmem : P.smem;
            int per_sm = 0;
            const cudaError_t oe =
                which == 0 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gkern, tpb, smem)
              : which == 1 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tkern, tpb, smem)
                           : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, tpb, smem);
            if (oe != cudaSuccess || per_sm < 1) {
                cudaGetLastError();
                return BB_ERR_UNSUPPORTED;
            }
            Launch LL = L;
            LL.total_tasks = which == 0 ? (int64_t)L.count * gtasks
                           : which == 1 ? (int64_t)L.count * ttasks : L.total_tasks;
            int64_t grid = (int64_t)nsm * per_sm;
            if (P.tune.sif > 0) grid = std::min<int64_t>(grid, P.tune.sif);
            else if (which == 0 && P.tune.dtype == BB_F64 && gsteps <= 3 * (int64_t)nsm)
                // FP64 group steps keep an SM's FP64 pipe busy: while the
                // stage's wavefront is short (few groups active at once) one
                // CTA per SM runs each group step at the SM's full rate
                grid = std::min<int64_t>(grid, nsm);
            grid = std::min<int64_t>(grid, LL.total_tasks);
            if (grid < 1) continue;
            if (!first && cudaMemsetAsync(&P.L.hdr->claim, 0, sizeof(int), st) != cudaSuccess)
                return BB_ERR_LAUNCH;
            first = false;
            cudaEvent_t* ev = (cudaEvent_t*)P.tune.ev_launch;
            const bool rec = ev && 2 * nlaunch + 1 < P.tune.ev_count;
            if (rec && cudaEventRecord(ev[2 * nlaunch], st) != cudaSuccess) return BB_ERR_LAUNCH;
            if (which == 0) gkern<<<(unsigned)grid, tpb, smem, st>>>(LL);
            else if (which == 1) tkern<<<(unsigned)grid, tpb, smem, st>>>(LL);
            else kern<<<(unsigned)grid, tpb, smem, st>>>(LL);
            if (cudaGetLastError() != cudaSuccess) return BB_ERR_LAUNCH;
            if (rec && cudaEventRecord(ev[2 * nlaunch + 1], st) != cudaSuccess) return BB_ERR_LAUNCH;
            if (P.tune.launch_log && nlaunch < P.tune.ev_count / 2)
                P.tune.launch_log[nlaunch] = stage * 4 + which;
            ++nlaunch;
        }
    }
    if (P.tune.ev_stop && cudaEventRecord(P.tune.ev_stop, st) != cudaSuccess) return BB_ERR_LAUNCH;
    return BB_OK;
}

template <typename TS, typename T>
int launch_all_t(const LaunchPlan& P, cudaStream_t st)
{
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const unsigned cols_grid = (unsigned)std::max<int64_t>(
        1, std::min<int64_t>((P.L.total_cols + 7) / 8, (int64_t)nsm * 16));
    pack_kernel<TS><<<cols_grid, 256, 0, st>>>(P.L);
    if (cudaGetLastError() != cudaSuccess) return BB_ERR_LAUNCH;
    if (P.max_stages > 0) {
        int rc;
        switch (maxm_for(P.tune.tw)) {
            case 5: rc = launch_stages<TS, T, 5>(P, st); break;
            case 9: rc = launch_stages<TS, T, 9>(P, st); break;
            case 17: rc = launch_stages<TS, T, 17>(P, st); break;
            default: rc = launch_stages<TS, T, 33>(P, st); break;
        }
        if (rc != BB_OK) return rc;
    }
    const unsigned ex_grid = (unsigned)std::max<int64_t>(
        1, std::min<int64_t>((P.L.total_cols + 255) / 256, (int64_t)nsm * 8));
    extract_kernel<TS><<<ex_grid, 256, 0, st>>>(P.L);
    return cudaGetLastError() == cudaSuccess ? BB_OK : BB_ERR_LAUNCH;
}

// enqueue: zero the counters, (upload the table), pack, bulge, extract
int enqueue(LaunchPlan* P, void* ws, const void* host_descs, cudaStream_t st)
{
    // panels that cannot fit this device's shared memory: refuse before any work
    int dev = 0, smem_optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return BB_ERR_LAUNCH;
    if (P->max_stages > 0 && P->smem > (size_t)smem_optin) return BB_ERR_UNSUPPORTED;
    // a group window larger than the device allows: fewer sweeps per CTA
    while (P->gsmem > (size_t)smem_optin && P->L.gK > 1) P->gsmem = group_smem_bytes(*P, --P->L.gK);
    if (P->gsmem > (size_t)smem_optin) { P->gsmem = 0; P->L.gK = 0; }
    while (P->tsmem > (size_t)smem_optin && P->L.team > 1) P->tsmem = team_smem_bytes(*P, --P->L.team);
    if (P->tsmem > (size_t)smem_optin) { P->tsmem = 0; P->L.team = 0; }
    bind_workspace(P, ws);
    if (cudaMemsetAsync(ws, 0, P->off_w, st) != cudaSuccess) return BB_ERR_LAUNCH;
    if (P->L.count > 1) {
        if (cudaMemcpyAsync((char*)ws + P->off_desc, host_descs, sizeof(Desc) * P->L.count,
                            cudaMemcpyHostToDevice, st) != cudaSuccess)
            return BB_ERR_LAUNCH;
    }
    switch (P->tune.dtype) {
        case BB_F64: return launch_all_t<double, double>(*P, st);
        case BB_F32: return launch_all_t<float, float>(*P, st);
        case BB_F16: return launch_all_t<__half, float>(*P, st);
        default: return launch_all_t<__nv_bfloat16, float>(*P, st);
    }
}

}  // namespace

// ------------------------------------------------------------------ C ABI

extern "C" {

int bb_default_tuning(int64_t n, int64_t b, int dtype, bb_tuning* out)
{
    if (!out) return BB_ERR_ARG;
    (void)n;
    out->tw = dtype == BB_F64 ? 16 : 32;     // one 128-byte line of FP64 / FP32 (the kernel's widest TW for half storage)
    out->tpb = 0;                             // per stage: two threads per panel row / column
    out->sweeps_in_flight = 0;
    out->flags = 0;
    out->timeout_s = 5.0;
    out->ev_start = nullptr;
    out->ev_stop = nullptr;
    out->group = 0;                           // default sweeps per CTA (kDefaultGroup)
    out->teams = 0;                           // default sweeps per CTA on the last stage
    out->ev_launch = nullptr;
    out->ev_count = 0;
    out->launch_log = nullptr;
    return BB_OK;
}

const char* bb_status_string(int code)
{
    switch (code) {
        case BB_OK: return "ok";
        case BB_ERR_ARG: return "invalid argument";
        case BB_ERR_ALLOC: return "workspace allocation failed";
        case BB_ERR_LAUNCH: return "kernel launch or CUDA call failed";
        case BB_ERR_TIMEOUT: return "device wait timed out";
        case BB_ERR_NONFINITE: return "non-finite input";
        case BB_ERR_WORKSPACE: return "workspace too small";
        case BB_ERR_UNSUPPORTED: return "unsupported configuration";
        default: return "unknown status";
    }
}

size_t band_to_bidiag_workspace_size(int64_t n, int64_t b, int dtype, const bb_tuning* tuning)
{
    bb_problem p = {n, b, (const void*)16, b + 1, (void*)16, (void*)16};
    LaunchPlan P;
    if (plan_launch(1, &p, dtype, tuning, &P) != BB_OK) return 0;
    return P.bytes;
}

size_t bb_shared_bytes(int64_t n, int64_t b, int dtype, const bb_tuning* tuning)
{
    bb_problem p = {n, b, (const void*)16, b + 1, (void*)16, (void*)16};
    LaunchPlan P;
    if (plan_launch(1, &p, dtype, tuning, &P) != BB_OK) return 0;
    return std::max(P.smem, std::max(P.gsmem, P.tsmem));
}

int band_to_bidiag_ex(int64_t n, int64_t b, int dtype, const void* band, int64_t ldab,
                      void* d_out, void* e_out, const bb_tuning* tuning, void* workspace,
                      size_t workspace_bytes, void* stream)
{
    bb_problem p = {n, b, band, ldab, d_out, e_out};
    LaunchPlan P;
    int rc = plan_launch(1, &p, dtype, tuning, &P);
    if (rc != BB_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    void* ws = workspace;
    bool own = false;
    if (ws) {
        if (workspace_bytes < P.bytes || ((uintptr_t)ws % kAlign) != 0) return BB_ERR_WORKSPACE;
    } else {
        if (cudaMallocAsync(&ws, P.bytes, st) != cudaSuccess) return BB_ERR_ALLOC;
        own = true;
    }
    rc = enqueue(&P, ws, nullptr, st);
    if (own) cudaFreeAsync(ws, st);
    return rc;
}

// ---- singular vectors: reflector store and back-transformation

}  // extern "C"

namespace {

// the tuning of the vectors path: as given, with the last stage on the
// per-sweep kernel (the team kernel does not store reflectors)
bb_tuning vectors_tuning(int64_t n, int64_t b, int dtype, const bb_tuning* t)
{
    bb_tuning v;
    if (t) v = *t;
    else bb_default_tuning(n, b, dtype, &v);
    v.teams = -1;
    return v;
}

// bytes of the reflector store: two slots per row-bulge of every stage
size_t refl_store_bytes(const LaunchPlan& P)
{
    const Desc& D = P.descs[0];
    int64_t k = 0;
    for (int st = 0; st < D.nstages; ++st) {
        const int bw = D.b - st * P.tune.tw, d = std::min(P.tune.tw, bw - 1);
        k += steps_before(D.n, bw, d, D.n);
    }
    const size_t es = P.tune.dtype == BB_F64 ? 8 : 4;
    return align_up((size_t)(2 * k) * (size_t)refl_stride(maxm_for(P.tune.tw)) * es);
}

template <typename T>
int backtransform_all(const LaunchPlan& P, T* q, int64_t ldq, T* p, int64_t ldp, cudaStream_t st)
{
    const Desc& D = P.descs[0];
    const int n = D.n, grid = (int)std::min<int64_t>(((int64_t)n * n + 255) / 256, 152 * 16);
    identity_kernel<T><<<grid, 256, 0, st>>>(q, ldq, n);
    identity_kernel<T><<<grid, 256, 0, st>>>(p, ldp, n);
    const T* refl = (const T*)P.L.refl;
    const dim3 g2((unsigned)((n + 31) / 32), 2);
    switch (maxm_for(P.tune.tw)) {
        case 5:
            backtransform_kernel<T, 5><<<g2, 32, 0, st>>>(n, D.b, P.tune.tw, refl, q, ldq, p, ldp);
            break;
        case 9:
            backtransform_kernel<T, 9><<<g2, 32, 0, st>>>(n, D.b, P.tune.tw, refl, q, ldq, p, ldp);
            break;
        case 17:
            backtransform_kernel<T, 17><<<g2, 32, 0, st>>>(n, D.b, P.tune.tw, refl, q, ldq, p, ldp);
            break;
        default:
            backtransform_kernel<T, 33><<<g2, 32, 0, st>>>(n, D.b, P.tune.tw, refl, q, ldq, p, ldp);
            break;
    }
    return cudaGetLastError() == cudaSuccess ? BB_OK : BB_ERR_LAUNCH;
}

}  // namespace

extern "C" {

size_t band_to_bidiag_vectors_workspace_size(int64_t n, int64_t b, int dtype, const bb_tuning* tuning)
{
    if (dtype != BB_F32 && dtype != BB_F64) return 0;
    const bb_tuning t = vectors_tuning(n, b, dtype, tuning);
    bb_problem p = {n, b, (const void*)16, b + 1, (void*)16, (void*)16};
    LaunchPlan P;
    if (plan_launch(1, &p, dtype, &t, &P) != BB_OK) return 0;
    return align_up(P.bytes) + refl_store_bytes(P);
}

int band_to_bidiag_vectors(int64_t n, int64_t b, int dtype, const void* band, int64_t ldab, void* d_out,
                           void* e_out, void* q_out, int64_t ldq, void* p_out, int64_t ldp,
                           const bb_tuning* tuning, void* workspace, size_t workspace_bytes, void* stream)
{
    if (dtype != BB_F32 && dtype != BB_F64) return dtype == BB_F16 || dtype == BB_BF16 ? BB_ERR_UNSUPPORTED : BB_ERR_ARG;
    if (!q_out || !p_out || ldq < n || ldp < n) return BB_ERR_ARG;
    const bb_tuning t = vectors_tuning(n, b, dtype, tuning);
    bb_problem p = {n, b, band, ldab, d_out, e_out};
    LaunchPlan P;
    int rc = plan_launch(1, &p, dtype, &t, &P);
    if (rc != BB_OK) return rc;
    const size_t need = align_up(P.bytes) + refl_store_bytes(P);
    cudaStream_t st = (cudaStream_t)stream;
    void* ws = workspace;
    bool own = false;
    if (ws) {
        if (workspace_bytes < need || ((uintptr_t)ws % kAlign) != 0) return BB_ERR_WORKSPACE;
    } else {
        if (cudaMallocAsync(&ws, need, st) != cudaSuccess) { cudaGetLastError(); return BB_ERR_ALLOC; }
        own = true;
    }
    P.L.refl = (char*)ws + align_up(P.bytes);
    rc = enqueue(&P, ws, nullptr, st);
    if (rc == BB_OK)
        rc = dtype == BB_F64 ? backtransform_all<double>(P, (double*)q_out, ldq, (double*)p_out, ldp, st)
                             : backtransform_all<float>(P, (float*)q_out, ldq, (float*)p_out, ldp, st);
    if (own) cudaFreeAsync(ws, st);
    return rc;
}

int band_to_bidiag(int64_t n, int64_t b, int dtype, const void* band, int64_t ldab, void* d_out,
                   void* e_out, void* stream)
{
    return band_to_bidiag_ex(n, b, dtype, band, ldab, d_out, e_out, nullptr, nullptr, 0, stream);
}

int bb_device_status(void* stream, int reset)
{
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return -BB_ERR_LAUNCH;
    unsigned v = 0;
    if (cudaMemcpyFromSymbol(&v, g_bb_status, sizeof(v)) != cudaSuccess) return -BB_ERR_LAUNCH;
    if (reset) {
        unsigned z = 0;
        if (cudaMemcpyToSymbol(g_bb_status, &z, sizeof(z)) != cudaSuccess) return -BB_ERR_LAUNCH;
    }
    return (int)v;
}

int bb_last_device_status(void* stream) { return bb_device_status(stream, 1); }

int band_to_bidiag_host(int64_t n, int64_t b, int dtype, const void* band, int64_t ldab,
                        void* d_out, void* e_out, const bb_tuning* tuning, void* stream)
{
    if (!band || !d_out || (n > 1 && !e_out) || n < 1 || ldab < b + 1) return BB_ERR_ARG;
    if (!dtype_ok(dtype)) return BB_ERR_ARG;
    const size_t es = (size_t)storage_size(dtype);
    const size_t band_bytes = align_up(es * (size_t)ldab * (size_t)n);
    const size_t d_bytes = align_up(es * (size_t)n);
    const size_t ws_bytes = band_to_bidiag_workspace_size(n, b, dtype, tuning);
    if (ws_bytes == 0) return BB_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    char* buf = nullptr;
    if (cudaMallocAsync((void**)&buf, band_bytes + 2 * d_bytes + ws_bytes, st) != cudaSuccess)
        return BB_ERR_ALLOC;
    char* dband = buf;
    char* dd = buf + band_bytes;
    char* de = dd + d_bytes;
    char* dws = de + d_bytes;
    int rc = BB_OK;
    if (cudaMemcpyAsync(dband, band, es * (size_t)ldab * (size_t)n, cudaMemcpyHostToDevice, st) != cudaSuccess)
        rc = BB_ERR_LAUNCH;
    if (rc == BB_OK)
        rc = band_to_bidiag_ex(n, b, dtype, dband, ldab, dd, n > 1 ? de : nullptr, tuning, dws, ws_bytes, st);
    if (rc == BB_OK && cudaMemcpyAsync(d_out, dd, es * (size_t)n, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        rc = BB_ERR_LAUNCH;
    if (rc == BB_OK && n > 1 &&
        cudaMemcpyAsync(e_out, de, es * (size_t)(n - 1), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        rc = BB_ERR_LAUNCH;
    cudaFreeAsync(buf, st);
    const int dev = bb_device_status(stream, 1);
    if (rc != BB_OK) return rc;
    if (dev < 0) return -dev;
    for (int code = 1; code < 16; ++code)
        if (dev & (1 << code)) return code;
    return BB_OK;
}

// ------------------------------------------------------------------- batch

struct bb_batch_plan {
    LaunchPlan P;
    Desc* pinned = nullptr;   // problem table for the host-to-device copy
};

bb_batch_plan* bb_batch_plan_create(int count, const bb_problem* problems, int dtype,
                                    const bb_tuning* tuning)
{
    bb_batch_plan* plan = new bb_batch_plan();
    if (plan_launch(count, problems, dtype, tuning, &plan->P) != BB_OK) {
        delete plan;
        return nullptr;
    }
    if (count > 1) {
        if (cudaMallocHost((void**)&plan->pinned, sizeof(Desc) * count) != cudaSuccess) {
            delete plan;
            return nullptr;
        }
        std::memcpy(plan->pinned, plan->P.descs.data(), sizeof(Desc) * count);
    }
    return plan;
}

size_t bb_batch_plan_workspace_size(const bb_batch_plan* plan) { return plan ? plan->P.bytes : 0; }

int bb_batch_execute(const bb_batch_plan* plan, void* workspace, size_t workspace_bytes, void* stream)
{
    if (!plan || !workspace) return BB_ERR_ARG;
    if (workspace_bytes < plan->P.bytes || ((uintptr_t)workspace % kAlign) != 0) return BB_ERR_WORKSPACE;
    LaunchPlan P = plan->P;   // the launch struct is bound to this workspace
    return enqueue(&P, workspace, plan->pinned, (cudaStream_t)stream);
}

int band_to_bidiag_batched(int count, const bb_problem* problems, int dtype, void* stream)
{
    LaunchPlan P;
    int rc = plan_launch(count, problems, dtype, nullptr, &P);
    if (rc != BB_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    void* ws = nullptr;
    if (cudaMallocAsync(&ws, P.bytes, st) != cudaSuccess) return BB_ERR_ALLOC;
    // the table goes from pageable memory, which the copy consumes before it returns
    rc = enqueue(&P, ws, count > 1 ? (const void*)P.descs.data() : nullptr, st);
    cudaFreeAsync(ws, st);
    return rc;
}

void bb_batch_plan_destroy(bb_batch_plan* plan)
{
    if (!plan) return;
    if (plan->pinned) cudaFreeHost(plan->pinned);
    delete plan;
}

// ------------------------------------------------------------ work model

int bb_schedule_counts(int64_t n64, int64_t b64, int tw, int64_t* stages_out, int64_t* steps_out,
                       double* flops_out, double* elems_out)
{
    return bb_stage_counts(n64, b64, tw, -1, stages_out, steps_out, flops_out, elems_out);
}

int bb_stage_counts(int64_t n64, int64_t b64, int tw, int stage, int64_t* stages_out,
                    int64_t* steps_out, double* flops_out, double* elems_out)
{
    if (n64 < 1 || b64 < 0 || tw < 1 || n64 >= PROG_STAGE) return BB_ERR_ARG;
    const int n = (int)n64;
    int b = clamp_b(n64, b64);
    int64_t stages = 0, steps = 0;
    double flops = 0.0, elems = 0.0;
    // cost of one row-bulge at block column c (generic data: both reflectors nontrivial)
    auto step_cost = [&](int bw, int d, int R, int s, double* f, double* e) {
        const int c = R + (bw - d) + s * bw;
        const int m = std::min(d + 1, n - c);
        const int r0 = (s == 0) ? R : c - bw;
        const int jmax = std::min(n - 1, c + m - 1 + bw);
        const int nr = c + m - r0, nc = jmax - c + 1;
        *f = 2.0 * (4.0 * (m - 1) + 10.0) + 4.0 * m * (nr - 1) + 4.0 * m * (nc - 1);
        *e = (double)nr * m + (double)m * nc - (double)m * m;
    };
    for (int bw = b; bw > 1;) {
        const int d = std::min(tw, bw - 1);
        ++stages;
        if (stage >= 0 && stages - 1 != stage) {   // only the requested stage
            bw -= d;
            continue;
        }
        for (int R = 0; R < n - 1; ++R) {
            const int c0 = R + bw - d;
            if (c0 >= n - 1) continue;
            const int ns = (n - 2 - c0) / bw + 1;
            steps += ns;
            // full steps: s >= 1 with c + d + bw <= n - 1
            int full_hi = (n - 1 - d - bw - c0) >= 0 ? (n - 1 - d - bw - c0) / bw : -1;
            full_hi = std::min(full_hi, ns - 1);
            double f, e;
            if (full_hi >= 1) {
                step_cost(bw, d, R, 1, &f, &e);
                flops += f * full_hi;
                elems += e * full_hi;
            }
            for (int s = 0; s < ns; ++s) {
                if (s >= 1 && s <= full_hi) continue;
                step_cost(bw, d, R, s, &f, &e);
                flops += f;
                elems += e;
            }
        }
        bw -= d;
    }
    if (stages_out) *stages_out = stages;
    if (steps_out) *steps_out = steps;
    if (flops_out) *flops_out = flops;
    if (elems_out) *elems_out = elems;
    return BB_OK;
}

}  // extern "C"

// ------------------------------------------------- allocation-free variant
//
// Some callers cannot allocate device memory at the point where they need the
// reduction: code running inside a CUDA stream capture that must not add
// allocation nodes, callers whose memory is fully reserved up front by their
// own pool or another framework's caching allocator, or host environments
// with no way to obtain or free a workspace.  band_to_bidiag_noalloc serves
// them: its scratch (counters and the working band) lives in one statically
// sized device array that the library defines, so the call allocates nothing.
//
// Cost and limits: every GPU that loads this library keeps the array
// (kNoAllocScratchBytes = 16 MiB) reserved until the process exits.  Problems
// whose workspace exceeds it are rejected.  All calls on a device share the one
// array, so calls whose GPU work may overlap (different streams, or
// concurrent host threads) race and corrupt each other's results; serialise
// them on one stream.  The counters at the front of the array are cleared on
// the stream by every call.

namespace {

constexpr size_t kNoAllocScratchBytes = 16u << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {};

// Device address of the scratch array for the current device (set up once per
// device, with that device current).  The host-side symbol is only a stand-in
// for the device array and must never be handed to a kernel.
void* noalloc_scratch_for_current_device()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) return nullptr;
        g_noalloc_ptr[dev] = p;
    }
    return g_noalloc_ptr[dev];
}

}  // namespace

extern "C" size_t band_to_bidiag_noalloc_max_bytes(void) { return kNoAllocScratchBytes; }

extern "C" int band_to_bidiag_noalloc(int64_t n, int64_t b, int dtype, const void* band,
                                      int64_t ldab, void* d_out, void* e_out, void* stream)
{
    bb_problem p = {n, b, band, ldab, d_out, e_out};
    LaunchPlan P;
    int rc = plan_launch(1, &p, dtype, nullptr, &P);
    if (rc != BB_OK) return rc;
    if (P.bytes > kNoAllocScratchBytes) return BB_ERR_WORKSPACE;
    void* ws = noalloc_scratch_for_current_device();
    if (!ws) return BB_ERR_LAUNCH;
    return enqueue(&P, ws, nullptr, (cudaStream_t)stream);
}
