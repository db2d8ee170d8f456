// Team kernel: the last bandwidth-reduction stage (bw -> 1, d = bw - 1) of
// arXiv 2510.12705, Section III (Algorithm 1 schedule, Algorithm 2
// row-bulge).  On this stage consecutive sweeps must stay two row-bulges
// apart (Section III-A: two right reflectors act on overlapping column sets,
// and a left reflector of sweep R+1 reaches the pivot of sweep R's row-bulge
// two steps ahead), so one CTA runs W consecutive sweeps side by side, one
// team of kTeamWarps warps per sweep (its first warp builds the reflectors,
// all of them apply them, two threads per row or column, with team barriers),
// and a last warp moves data.
//
// Shared memory holds a circular band window of C columns: matrix column x in
// slot x mod C, band offsets i - x in [-(2bw-1), bw-1] (the only ones this
// stage touches) at slot * P + (i - x + 2bw - 1).  Team j (sweep R0 + j)
// processes its row-bulges in order on the window and waits only on team j-1
// through shared-memory counters with acquire / release semantics: step s
// starts once team j-1 completed step s+1, and the last column of its left
// reflector waits until team j-1 applied the right reflector of step s+2 (the
// per-sweep protocol, checked against every footprint on the host).
// The IO warp owns the columns: it loads a column once the previous group has
// released it (global progress word = first column not yet released) and its
// slot is free, and it stores and releases a column once every team of the
// group is past it.  Column ownership thus passes from group to group; within
// a group the window is shared.
#pragma once

#include "bb_device.cuh"

namespace bb {

// One lane: spin until *p >= target (shared memory).  Gives up (sets the
// error and abort words) when nothing changed for timeout_ns or another CTA
// aborted.
// The polls are relaxed; one acquire load follows once the target is seen.
__device__ __forceinline__ bool wait_shared(const int* p, int target, Header* hdr,
                                            unsigned long long timeout_ns)
{
    int last = ld_relaxed_shared(p);
    if (last >= target) { (void)ld_acquire_shared(p); return true; }
    unsigned long long t_last = global_ns();
    for (int it = 1;; ++it) {
        if (it > 32) __nanosleep(32);
        const int v = ld_relaxed_shared(p);
        if (v >= target) { (void)ld_acquire_shared(p); return true; }
        if ((it & 15) == 0) {
            if (ld_relaxed(&hdr->abort)) return false;
            const unsigned long long now = global_ns();
            if (v != last) { last = v; t_last = now; continue; }
            if (now - t_last > timeout_ns) {
                atomicOr(&hdr->err, 1 << 4 /* BB_ERR_TIMEOUT */);
                atomicExch(&hdr->abort, 1);
                return false;
            }
        }
    }
}

// window geometry for teams W on a last stage of bandwidth bw
__host__ __device__ __forceinline__ int team_pitch(int bw) { const int p = 3 * bw - 1; return p + (p & 1); }
__host__ __device__ __forceinline__ int team_cols(int bw, int W) { return (2 * W + 3) * bw; }
__host__ __device__ __forceinline__ int team_scratch_elems(int maxm)
{
    // per team: vR, vL (maxm each), tb (8), xb (maxm + 1), ts (64), column bases (2 maxm, ints as T)
    return (2 * maxm + 8 + maxm + 1 + 64 + 2 * maxm + 3) & ~3;
}
__host__ __device__ __forceinline__ int team_smem_elems(int bw, int W, int maxm)
{
    return team_cols(bw, W) * team_pitch(bw) + W * team_scratch_elems(maxm);
}

// warps per team (one per SM sub-partition)
constexpr int kTeamWarps = 4;

// Team of nt threads (tt = this thread's index in the team): reflector
// (v, tau) from the right on window rows [r_lo, r_hi] of the m columns whose
// slot bases are cb[0..m) (row i of column c+t at cb[t] + i - (c + t)).  Two
// threads per row: thread p of a pair takes the entries [p H, p H + H) and one
// shuffle combines the halves.  Loads go to clamped, always valid addresses;
// v is zero beyond m, so the extra terms vanish, and only the stores are
// guarded.  Every thread of the team runs the same number of passes.
template <typename T, int MAXM>
__device__ __forceinline__ void team_apply_right(T* win, const int* cb, int c, int m, int r_lo,
                                                 int r_hi, const T* v, T tau, int tt, int nt)
{
    constexpr int H = (MAXM + 1) / 2;
    const int k0 = (tt & 1) * H, np = nt >> 1;
    const int nrows = r_hi - r_lo + 1;
    for (int base = 0; base < nrows; base += np) {
        const int ri = base + (tt >> 1);
        const bool act = ri < nrows;
        const int r = r_lo + (act ? ri : nrows - 1);
        T a[H];
        T w = (T)0;
#pragma unroll
        for (int i = 0; i < H; ++i) {
            const int t = k0 + i, tc = t < m ? t : m - 1;
            a[i] = win[cb[tc] + r - (c + tc)];
            if (t < MAXM) w = fma(a[i], v[t], w);
        }
        w += __shfl_xor_sync(FULL, w, 1);
        const T tw = tau * w;
        if (act) {
#pragma unroll
            for (int i = 0; i < H; ++i) {
                const int t = k0 + i;
                if (t < m) win[cb[t] + r - (c + t)] = fma(-tw, v[t], a[i]);
            }
        }
    }
}

// Team: reflector (v, tau) from the left on rows [c, c+m) of columns
// [x_lo, x_hi] (column c+k at cb[k]); two threads per column as above.
template <typename T, int MAXM>
__device__ __forceinline__ void team_apply_left(T* win, const int* cb, int c, int m, int x_lo,
                                                int x_hi, const T* v, T tau, int tt, int nt)
{
    constexpr int H = (MAXM + 1) / 2;
    const int k0 = (tt & 1) * H, np = nt >> 1;
    const int ncols = x_hi - x_lo + 1;
    for (int base = 0; base < ncols; base += np) {
        const int xi = base + (tt >> 1);
        const bool act = xi < ncols;
        const int x = x_lo + (act ? xi : ncols - 1);
        T* col = win + cb[x - c] + (c - x);     // row c + t at col[t]
        T a[H];
        T w = (T)0;
#pragma unroll
        for (int i = 0; i < H; ++i) {
            const int t = k0 + i;
            a[i] = col[t < m ? t : m - 1];
            if (t < MAXM) w = fma(a[i], v[t], w);
        }
        w += __shfl_xor_sync(FULL, w, 1);
        const T tw = tau * w;
        if (act) {
#pragma unroll
            for (int i = 0; i < H; ++i) {
                const int t = k0 + i;
                if (t < m) col[t] = fma(-tw, v[t], a[i]);
            }
        }
    }
}

template <typename TS, typename T, int MAXM>
__global__ void __launch_bounds__(32 * (4 * kTeamWarps + 1)) team_kernel(Launch L)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_task[2];
    __shared__ int tprog[16];     // per team: 2 * steps done (+1: right reflector of the next done)
    __shared__ int s_loaded;      // columns < s_loaded are in the window
    __shared__ int s_abort;
    __shared__ int s_tok[16][2];  // per team: results of its leader's waits (two slots in turn,
                                  // so a slow reader never sees the next result)
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int W = ((blockDim.x >> 5) - 1) / kTeamWarps;   // teams; warp W * kTeamWarps moves data
    const int IOW = W * kTeamWarps;
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
        if (bw - d != 1) continue;                 // not the last stage of this problem
        const int nact = n - 2;                    // sweeps with a row-bulge
        if (nact <= 0 || g >= (nact + W - 1) / W) continue;
        const int R0 = g * W;
        const int kk = min(W, nact - R0);
        const int P = team_pitch(bw), C = team_cols(bw, W);
        T* const win = (T*)smem_raw;
        TS* const Wg = (TS*)L.wbase + D.w_off;
        const int ldw = D.ldw, top = D.top;
        int* const my = L.prog + D.prog_off + (int64_t)g * ps;
        const int* const pred = g > 0 ? my - ps : nullptr;
        const bool stall = (L.flags & BB_FLAG_INJECT_STALL) && stage == 0 && g == 0;
        if (tid < 16) tprog[tid] = 0;
        if (tid == 0) { s_loaded = R0 + 1; s_abort = 0; }
        __syncthreads();

        if (warp == IOW) {
            // ---------------------------------------------------------- IO warp
            // lane j < kk follows team j: the first column of its next row-bulge
            const int nsj = lane < kk ? sweep_steps(n, bw, d, R0 + lane) : 0;
            int ld = R0 + 1, st = R0 + 1;          // next column to load / to store
            int avail = g == 0 ? n : 0;
            unsigned long long t_last = global_ns();
            bool ok = true;
            while (st < n) {
                bool progress = false;
                // release: columns left of every team's next row-bulge (after the
                // first steps the last team is the leftmost; at the start the
                // earlier teams are one column further left each)
                int rel = n;
                if (lane < kk) {
                    const int pj = ld_relaxed_shared(&tprog[lane]) >> 1;
                    if (pj < nsj) rel = R0 + lane + 1 + pj * bw;
                }
                rel = __reduce_min_sync(FULL, rel);
                const int st_to = min(rel, ld);
                if (st_to > st) {
                    // the teams' updates of these columns: acquire once
                    if (lane < kk) (void)ld_acquire_shared(&tprog[lane]);
                    __syncwarp();
                    for (int x = st; x < st_to; ++x) {          // one column segment at a time
                        const T* src = win + (x % C) * P;
                        TS* dst = Wg + (int64_t)x * ldw + (top - 2 * bw + 1);
                        for (int o = lane; o < 3 * bw - 1; o += 32) panel_to_band<TS, T>(dst + o, src[o]);
                    }
                    __syncwarp();
                    st = st_to;
                    if (lane == 0 && !stall) st_release(my, base + st);
                    progress = true;
                }
                // load: columns the previous group released whose slots are free
                if (ld < n) {
                    if (avail <= ld && g > 0) {
                        // relaxed poll; one acquire once new columns are released
                        int a = 0;
                        if (lane == 0) {
                            a = ld_relaxed(pred) - base;
                            if (a > ld) a = ld_acquire(pred) - base;
                        }
                        avail = __shfl_sync(FULL, a, 0);
                    }
                    const int ld_to = min(min(avail, n), min(st + C, ld + bw));
                    if (ld_to > ld) {
                        for (int x = ld; x < ld_to; ++x) {
                            T* dst = win + (x % C) * P;
                            const TS* src = Wg + (int64_t)x * ldw + (top - 2 * bw + 1);
                            for (int o = lane; o < 3 * bw - 1; o += 32) band_to_panel<TS, T>(dst + o, src + o);
                        }
                        cp_async_wait_all();
                        __syncwarp();
                        ld = ld_to;
                        if (lane == 0) st_release_shared(&s_loaded, ld);
                        progress = true;
                    }
                }
                if (progress) { t_last = global_ns(); continue; }
                int ab = 0;
                if (lane == 0) {
                    __nanosleep(100);
                    ab = ld_relaxed(&L.hdr->abort) || ld_relaxed_shared(&s_abort);
                    if (!ab && global_ns() - t_last > L.timeout_ns) {
                        atomicOr(&L.hdr->err, 1 << 4 /* BB_ERR_TIMEOUT */);
                        atomicExch(&L.hdr->abort, 1);
                        ab = 1;
                    }
                }
                if (__shfl_sync(FULL, ab, 0)) { ok = false; break; }
            }
            if (!ok && lane == 0) st_release_shared(&s_abort, 1);
        } else if (warp < IOW && warp / kTeamWarps < kk) {
            // ------------------------------------------------------------- team
            const int j = warp / kTeamWarps, R = R0 + j;
            const int tt = tid - j * kTeamWarps * 32, nt = kTeamWarps * 32;
            const bool lead = (warp % kTeamWarps) == 0;   // builds the reflectors, takes the waits
            const int bar = 1 + j;                         // named barrier of this team
            const int ns = sweep_steps(n, bw, d, R);
            const int nsp = j > 0 ? sweep_steps(n, bw, d, R - 1) : 0;
            T* const scr = win + C * P + j * team_scratch_elems(MAXM);
            T* const vR = scr;
            T* const vL = vR + MAXM;
            T* const tb = vL + MAXM;            // tau, beta, vs (right) | tau, beta, vs (left) at +4
            T* const xb = tb + 8;
            T* const ts = xb + MAXM + 1;
            int* const cb = (int*)(ts + 64);    // slot bases of the row-bulge's columns
            bool ok = true;
            int tk = 0;                         // waits so far: slot tk & 1 of s_tok[j]
            for (int s = 0; s < ns && ok; ++s) {
                const int c = R + 1 + s * bw;
                const int m = min(d + 1, n - c);
                const int r0 = s == 0 ? R : c - bw;
                const int jmax = min(n - 1, c + m - 1 + bw);
                // wait: team j-1 completed step s+1 (team 0: the right panel's columns loaded)
                if (lead && lane == 0)
                    s_tok[j][tk & 1] = j > 0 ? (int)wait_shared(&tprog[j - 1], 2 * min(s + 2, nsp), L.hdr, L.timeout_ns)
                                     : (int)wait_shared(&s_loaded, c + m, L.hdr, L.timeout_ns);
                for (int k = tt; k <= jmax - c; k += nt) cb[k] = ((c + k) % C) * P + 2 * bw - 1;
                bar_sync_n(bar, nt);
                if (!s_tok[j][tk++ & 1]) { ok = false; break; }
                // right reflector from row r0, columns c .. c+m-1
                if (lead) {
                    for (int t = lane; t < m; t += 32) xb[t] = win[cb[t] + r0 - (c + t)];
                    __syncwarp();
                    fast_reflector<T, MAXM>(m, xb, vR, tb);
                    __syncwarp();
                    for (int t = lane; t < m; t += 32) win[cb[t] + r0 - (c + t)] = t == 0 ? tb[1] : (T)0;
                }
                bar_sync_n(bar, nt);
                team_apply_right<T, MAXM>(win, cb, c, m, r0 + 1, c + m - 1, vR, tb[0], tt, nt);
                bar_sync_n(bar, nt);
                if (lead && lane == 0) st_release_shared(&tprog[j], 2 * s + 1);
                // left reflector from column c, rows c .. c+m-1
                if (lead) {
                    fast_reflector<T, MAXM>(m, win + cb[0], vL, tb + 4);
                    __syncwarp();
                    for (int t = lane; t < m; t += 32) win[cb[0] + t] = t == 0 ? tb[5] : (T)0;
                    // the last column c + d + bw is shared with team j-1's row-bulge s+2
                    const int xt = c + d + bw;
                    const bool tail = xt <= jmax;
                    if (lane == 0) {
                        int w_ok = 1;
                        if (j == 0) w_ok = (int)wait_shared(&s_loaded, jmax + 1, L.hdr, L.timeout_ns);
                        else if (tail)
                            w_ok = (int)wait_shared(&tprog[j - 1], s + 2 < nsp ? 2 * (s + 2) + 1 : 2 * nsp,
                                                    L.hdr, L.timeout_ns);
                        s_tok[j][tk & 1] = w_ok;
                    }
                }
                bar_sync_n(bar, nt);
                if (!s_tok[j][tk++ & 1]) { ok = false; break; }
                team_apply_left<T, MAXM>(win, cb, c, m, c + 1, jmax, vL, tb[4], tt, nt);
                bar_sync_n(bar, nt);
                // a sweep can be one row-bulge shorter than its predecessor: its
                // completion is published once the predecessor is complete, so
                // a completed sweep vouches for the whole chain before it
                if (lead && lane == 0) {
                    int w_ok = 1;
                    if (s == ns - 1 && j > 0) w_ok = (int)wait_shared(&tprog[j - 1], 2 * nsp, L.hdr, L.timeout_ns);
                    if (w_ok) st_release_shared(&tprog[j], 2 * (s + 1));
                    s_tok[j][tk & 1] = w_ok;
                }
                bar_sync_n(bar, nt);
                if (!s_tok[j][tk++ & 1]) { ok = false; break; }
            }
            if (!ok && lead && lane == 0) st_release_shared(&s_abort, 1);
        }
        __syncthreads();
        if (s_abort || ld_relaxed(&L.hdr->abort)) break;
    }
}

}  // namespace bb
