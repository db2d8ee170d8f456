// Device building blocks of the band -> bidiagonal reducer (sm_103a).
//
// Working storage: every problem owns a band-with-fill buffer in column-major
// band layout, element (i, j) at W[(i - j + top) + j * ldw], top = b + TW,
// ldw >= b + 2 TW + 1 (the band of height BW + 2 TW of Section V).  A column's
// band segment is contiguous, so the right panel of a row-bulge (rows x
// TW+1 columns) and the left panel (TW+1 rows x columns) are both runs of
// contiguous column segments.  Shared-working-buffer traffic goes through L2
// (ld/st .cg), the level on which concurrent sweeps hand data to each other.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace bb {

constexpr unsigned FULL = 0xffffffffu;
constexpr int PROG_STAGE = 1 << 20;   // progress word = stage * PROG_STAGE + steps done

// --------------------------------------------------------------- memory ops
template <typename T> __device__ __forceinline__ T ldcg(const T* p) { return __ldcg(p); }
template <typename T> __device__ __forceinline__ void stcg(T* p, T v) { __stcg(p, v); }

__device__ __forceinline__ int ld_acquire(const int* p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(int* p, int v)
{
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_relaxed(const int* p)
{
    int v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// ------------------------------------------------------------ workspace
// header words of a launch (one per batch)
struct Header {
    int claim;      // next task to hand out
    int abort;      // set when any wait ran out: every CTA stops
    int err;        // device error bits (1 << BB_ERR_*)
    int pad[5];
};

// one problem of a launch (device side)
struct Desc {
    int n;           // order
    int b;           // bandwidth after clamping to n-1
    int b_in;        // bandwidth of the caller's storage
    int nstages;     // bandwidth-reduction stages
    int ldw;         // working-band leading dimension
    int top;         // row offset of the diagonal in a working column
    int64_t w_off;   // element offset of the working band in the workspace
    int64_t prog_off;// int offset of the per-sweep progress words
    int64_t sweep_prefix;  // sum of (n - 1) over the previous problems
    int64_t col_prefix;    // sum of n over the previous problems
    const void* band;
    int64_t ldab;
    void* d;
    void* e;
};

struct Launch {
    const Desc* descs;    // device table (batched) or nullptr
    Desc single;          // the problem when descs == nullptr
    int count;            // problems
    int tw;               // inner tilewidth
    int64_t sweeps_per_stage;  // sum over problems of (n - 1)
    int64_t total_tasks;       // max_stages * sweeps_per_stage
    int64_t total_cols;        // sum over problems of n
    void* wbase;          // working bands
    int* prog;            // progress words
    int* stage_done;      // per problem: completed sweeps over all stages
    Header* hdr;
    unsigned long long timeout_ns;
    int flags;
    int rp_rows;          // shared-memory right panel rows (>= max b + TW + 1)
    int lp_cols;          // shared-memory left panel columns (>= max b + TW + 1)
};

__device__ __forceinline__ const Desc& desc_of(const Launch& L, int q)
{
    return L.descs ? L.descs[q] : L.single;
}

// problem index of a global sweep / column index (binary search over prefixes)
__device__ __forceinline__ int find_problem_by_sweep(const Launch& L, int64_t r)
{
    if (!L.descs) return 0;
    int lo = 0, hi = L.count - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (L.descs[mid].sweep_prefix <= r) lo = mid; else hi = mid - 1;
    }
    return lo;
}
__device__ __forceinline__ int find_problem_by_col(const Launch& L, int64_t c)
{
    if (!L.descs) return 0;
    int lo = 0, hi = L.count - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (L.descs[mid].col_prefix <= c) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// stage geometry: stage i reduces bw = b - i*tw to bw - d, d = min(tw, bw - 1)
__device__ __forceinline__ int stage_bw(int b, int tw, int i) { return b - i * tw; }
__device__ __forceinline__ int stage_d(int bw, int tw) { return tw < bw - 1 ? tw : bw - 1; }
// row-bulges of sweep R in stage (bw, d)
__device__ __forceinline__ int sweep_steps(int n, int bw, int d, int R)
{
    int c0 = R + (bw - d);
    return (c0 >= n - 1) ? 0 : (n - 2 - c0) / bw + 1;
}

// --------------------------------------------------------- warp reductions
__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(FULL, v, o));
    return v;
}

// ------------------------------------------------------ reflector generation
// Warp-cooperative Householder generation with the xLARFG contract, in FP64
// whatever the storage type: x (length m <= 64, stride xs, in shared memory)
// gives beta, tau and v (v[0] = 1) such that (I - tau v v^T) x = (beta, 0..0).
// tau = 0 when x(1:) == 0.  The norm is scaled by max|x_k|; when |beta| is
// below safmin the vector is rescaled by 1/safmin (up to 20 times) as in the
// documented LAPACK algorithm.  Called by all 32 lanes of one warp.
template <typename T>
__device__ void warp_reflector(int m, const T* x, int xs, T* v, T* tau_beta)
{
    const int lane = threadIdx.x & 31;
    const double safmin = 2.2250738585072014e-308 / 2.220446049250313e-16;
    double x0 = (lane < m) ? (double)x[lane * xs] : 0.0;
    double x1 = (lane + 32 < m) ? (double)x[(lane + 32) * xs] : 0.0;
    double alpha = __shfl_sync(FULL, x0, 0);
    double t0 = (lane >= 1) ? x0 : 0.0;   // tail x(1:)
    double scale = warp_max(fmax(fabs(t0), fabs(x1)));
    if (m <= 1 || scale == 0.0) {
        if (lane < m) v[lane] = (T)(lane == 0 ? 1.0 : 0.0);
        if (lane + 32 < m) v[lane + 32] = (T)0;
        if (lane == 0) { tau_beta[0] = (T)0; tau_beta[1] = (T)alpha; }
        return;
    }
    double q0 = t0 / scale, q1 = x1 / scale;
    double xnorm = scale * sqrt(warp_sum(q0 * q0 + q1 * q1));
    double beta = hypot(alpha, xnorm);
    if (alpha >= 0.0) beta = -beta;
    int knt = 0;
    if (fabs(beta) < safmin) {
        const double rs = 1.0 / safmin;
        do {
            ++knt;
            t0 *= rs; x1 *= rs; beta *= rs; alpha *= rs;
        } while (fabs(beta) < safmin && knt < 20);
        scale = warp_max(fmax(fabs(t0), fabs(x1)));
        q0 = t0 / scale; q1 = x1 / scale;
        xnorm = scale * sqrt(warp_sum(q0 * q0 + q1 * q1));
        beta = hypot(alpha, xnorm);
        if (alpha >= 0.0) beta = -beta;
    }
    const double tau = (beta - alpha) / beta;
    const double scal = 1.0 / (alpha - beta);
    if (lane < m) v[lane] = (T)(lane == 0 ? 1.0 : t0 * scal);
    if (lane + 32 < m) v[lane + 32] = (T)(x1 * scal);
    for (int j = 0; j < knt; ++j) beta *= safmin;
    if (lane == 0) { tau_beta[0] = (T)tau; tau_beta[1] = (T)beta; }
}

// ----------------------------------------------------------- bounded waits
// Spin until *addr >= target.  Gives up (sets the error and abort words and
// returns false) when the watched word has not changed for timeout_ns, or
// when another CTA aborted.  Called by one thread.
__device__ bool wait_at_least(const int* addr, int target, Header* hdr,
                              unsigned long long timeout_ns)
{
    int last = ld_acquire(addr);
    if (last >= target) return true;
    unsigned long long t_last = global_ns();
    unsigned backoff = 32;
    for (;;) {
        __nanosleep(backoff);
        if (backoff < 256) backoff <<= 1;
        int v = ld_acquire(addr);
        if (v >= target) return true;
        if (ld_relaxed(&hdr->abort)) return false;
        unsigned long long now = global_ns();
        if (v != last) { last = v; t_last = now; backoff = 32; continue; }
        if (now - t_last > timeout_ns) {
            atomicOr(&hdr->err, 1 << 4 /* BB_ERR_TIMEOUT */);
            atomicExch(&hdr->abort, 1);
            return false;
        }
    }
}

}  // namespace bb
