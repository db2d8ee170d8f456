// Device building blocks of the band -> bidiagonal reducer (sm_103a).
//
// Working storage: every problem owns a band-with-fill buffer in column-major
// band layout, element (i, j) at W[(i - j + top) + j * ldw], top = b + TW,
// ldw >= b + 2 TW + 1 (the band of height BW + 2 TW of Section IV).  A column's
// band segment is contiguous, so the right panel of a row-bulge (rows x
// TW+1 columns) and the left panel (TW+1 rows x columns) are both runs of
// contiguous column segments.  Shared-working-buffer traffic goes through L2
// (ld/st .cg), the level on which concurrent sweeps hand data to each other.
#pragma once

#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

namespace bb {

constexpr unsigned FULL = 0xffffffffu;
constexpr int PROG_STAGE = 1 << 20;   // progress word = stage * PROG_STAGE + 2 * row-bulges done (+1: right half of the next)

// --------------------------------------------------------------- memory ops
template <typename T> __device__ __forceinline__ T ldcg(const T* p) { return __ldcg(p); }
template <typename T> __device__ __forceinline__ void stcg(T* p, T v) { __stcg(p, v); }

// Asynchronous global -> shared copy of one element (cp.async, 4 or 8 bytes),
// completed by cp_async_wait_all().  The data it reads was published by other
// SMs through a release / acquire pair that one thread of the CTA observed
// before a barrier, which orders these reads after it.
template <typename T> __device__ __forceinline__ void cp_async_elem(T* smem, const T* gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    if constexpr (sizeof(T) == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s), "l"(gmem) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Storage type TS of the working band and compute type T of the panels: equal
// for the FP64 and FP32 forms; FP16 / BF16 storage computes in FP32.
template <typename T> __device__ __forceinline__ float to_float(T v) { return (float)v; }
template <> __device__ __forceinline__ float to_float<__half>(__half v) { return __half2float(v); }
template <> __device__ __forceinline__ float to_float<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

template <typename TS, typename T> __device__ __forceinline__ TS to_storage(T v) { return (TS)v; }
template <> __device__ __forceinline__ __half to_storage<__half, float>(float v) { return __float2half_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat16 to_storage<__nv_bfloat16, float>(float v)
{
    return __float2bfloat16_rn(v);
}

// one element of the working band (L2, bypassing L1) into a panel: an
// asynchronous copy when no conversion is needed, else a load and a convert
template <typename TS, typename T> __device__ __forceinline__ void band_to_panel(T* smem, const TS* g)
{
    if constexpr (sizeof(TS) == sizeof(T)) cp_async_elem(smem, (const T*)g);
    else *smem = (T)to_float(__ldcg(g));
}
template <typename TS, typename T> __device__ __forceinline__ void panel_to_band(TS* g, T v)
{
    if constexpr (sizeof(TS) == sizeof(T)) __stcg((T*)g, v);
    else __stcg(g, to_storage<TS, T>(v));
}

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
__device__ __forceinline__ int ld_acquire_shared(const int* p)
{
    int v;
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ld.acquire.cta.shared::cta.b32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ int ld_relaxed_shared(const int* p)
{
    int v;
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ld.relaxed.cta.shared::cta.b32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_shared(int* p, int v)
{
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("st.release.cta.shared::cta.b32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}

// named barriers: id 0 is __syncthreads; n threads (a multiple of 32) take part
__device__ __forceinline__ void bar_arrive(int id, int n)
{
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(n) : "memory");
}
__device__ __forceinline__ void bar_sync_n(int id, int n)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
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
    int64_t prog_off;// int offset of the per-sweep progress words (stride prog_stride)
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
    int64_t total_tasks;       // tasks of one stage launch: count * max(n - 1)
    int64_t total_cols;        // sum over problems of n
    void* wbase;          // working bands
    int* prog;            // progress words, one per sweep every prog_stride ints
    int prog_stride;      // 32 (one 128-byte line per sweep) for a single problem
    int* stage_done;      // per problem: completed sweeps over all stages
    Header* hdr;
    unsigned long long timeout_ns;
    int flags;
    int rp_rows;          // shared-memory right panel rows (>= max b + TW + 1)
    int lp_cols;          // shared-memory left panel columns (>= max b + TW + 1)
    int stage;            // bandwidth-reduction stage of this launch
    int gK;               // sweeps per CTA of the group kernel (0: every stage runs
                          // one sweep per CTA); the per-sweep kernel skips the
                          // problems the group kernel takes on this stage
    int team;             // sweeps per CTA of the team kernel on the last stage
                          // (0: the per-sweep kernel runs it)
    void* refl;           // reflector store of a single problem (compute type; nullptr: none):
                          // slot 2 k + side (0 right, 1 left) of row-bulge k holds
                          // v[0 .. MAXM) then tau, REFL_STRIDE(MAXM) elements a slot
    int64_t refl_base;    // row-bulges of the stages before this launch's stage
};

// elements of one reflector slot in the store: v (MAXM) and tau, rounded to 4
__host__ __device__ constexpr int refl_stride(int maxm) { return (maxm + 1 + 3) & ~3; }

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
// sum_{t=0}^{T} floor(t / bw) for T >= -1
__host__ __device__ __forceinline__ int64_t floor_sum(int64_t T, int64_t bw)
{
    if (T < 0) return 0;
    const int64_t q = T / bw, r = T - q * bw;
    return bw * q * (q - 1) / 2 + q * (r + 1);
}
// row-bulges of the sweeps before sweep R in stage (bw, d) of an order-n
// problem: sweep R' has floor((a - R') / bw) + 1 of them for R' <= a, where
// a = n - 2 - (bw - d), and none after (the count sweep_steps gives)
__host__ __device__ __forceinline__ int64_t steps_before(int n, int bw, int d, int64_t R)
{
    const int64_t a = (int64_t)n - 2 - (bw - d);
    const int64_t rc = R < a + 1 ? R : a + 1;
    if (rc <= 0) return 0;
    return rc + floor_sum(a, bw) - floor_sum(a - rc, bw);
}

// Store a reflector built by one warp (v[0 .. m) in shared memory, and tau)
// into its slot of the reflector store: slot k of a launch's stage is row-bulge
// refl_base + steps_before(n, bw, d, R) + s, side 0 (right) or 1 (left).
template <typename T, int MAXM>
__device__ __forceinline__ void warp_store_reflector(const Launch& L, int n, int bw, int d, int R, int s,
                                                     int side, int m, const T* v, T tau)
{
    const int lane = threadIdx.x & 31;
    const int64_t k = L.refl_base + steps_before(n, bw, d, R) + s;
    T* slot = (T*)L.refl + (2 * k + side) * (int64_t)refl_stride(MAXM);
    for (int t = lane; t < m; t += 32) slot[t] = v[t];
    if (lane == 0) slot[MAXM] = tau;
}

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
// Reciprocal and reciprocal square root in FP64 by Newton-Raphson iteration
// from an FP32 starting value (two steps: ~2^-23 -> ~2^-46 -> full
// precision).  The argument must be a positive normal number within the FP32
// range, which the power-of-two scaling in warp_reflector guarantees.
// STEPS = 1 reaches ~2^-46 (enough for results rounded to FP32), 2 full FP64.
template <int STEPS>
__device__ __forceinline__ double newton_rcp(double x)
{
    double y = (double)(1.0f / (float)x);
#pragma unroll
    for (int i = 0; i < STEPS; ++i) {
        const double e = fma(-x, y, 1.0);
        y = fma(y, e, y);
    }
    return y;
}
template <int STEPS>
__device__ __forceinline__ double newton_rsqrt(double x)
{
    double y = (double)rsqrtf((float)x);
    const double hx = 0.5 * x;
#pragma unroll
    for (int i = 0; i < STEPS; ++i) {
        const double e = fma(-hx * y, y, 0.5);     // (1 - x y^2) / 2
        y = fma(y, e, y);
    }
    return y;
}

// Warp-cooperative Householder generation with the xLARFG contract, in FP64
// whatever the storage type.  x (length m <= 64, contiguous in shared memory)
// gives beta, tau and v (v[0] = 1) with (I - tau v v^T) x = (beta, 0..0);
// tau = 0 when x(1:) == 0, and beta = -sign(alpha) ||x|| with sign(+-0) = +1.
// Overflow and underflow are avoided by scaling x by the power of two sc that
// brings its largest entry into [1, 4) (exact; it subsumes LAPACK's 1/safmin
// rescaling loop).  With the scaled vector t = sc x, s2 = ||t||^2 and
// r = 1/sqrt(s2):
//   beta = -sign(alpha) s2 r / sc,   tau = 1 + |t0| r,
//   v_k = vs t_k with vs = sign(alpha) / (|t0| + s2 r).
// Two entry points so that other warps can work while the FP64 chain runs:
//   reflector_scale: writes t (in T) to ts[] and returns after that;
//   reflector_finish: writes v[], tb = {tau, beta, vs}.
// Both are called by all 32 lanes of one warp, in this order.
struct ReflScale {
    double t0, y, a, alpha, inv_hi, inv_lo;   // a = scaled alpha
    bool zero;   // tail of x is zero: H = I
};

template <typename T>
__device__ __forceinline__ ReflScale reflector_scale(int m, const T* x, T* ts)
{
    const int lane = threadIdx.x & 31;
    ReflScale r;
    const double x0 = (lane < m) ? (double)x[lane] : 0.0;
    const double x1 = (lane + 32 < m) ? (double)x[lane + 32] : 0.0;
    r.alpha = __shfl_sync(FULL, x0, 0);
    const double tl = (lane >= 1) ? x0 : 0.0;   // tail x(1:)
    r.zero = (m <= 1) || !__any_sync(FULL, tl != 0.0 || x1 != 0.0);
    auto expo = [](double a) { return (unsigned)(__double_as_longlong(a) >> 52) & 0x7ffu; };
    unsigned ef = max(max(expo(x0), expo(x1)), 0u);
    ef = __reduce_max_sync(FULL, ef);
    double sc_hi, sc_lo = 1.0;
    r.inv_lo = 1.0;
    if (ef == 0) {
        sc_hi = 0x1p1022; sc_lo = 0x1p52; r.inv_hi = 0x1p-1022; r.inv_lo = 0x1p-52;
    } else {
        const unsigned es = min(ef, 2045u);
        sc_hi = __longlong_as_double((long long)(2046u - es) << 52);   // 2^(1023 - es)
        r.inv_hi = __longlong_as_double((long long)es << 52);          // 2^(es - 1023)
    }
    const double s0 = x0 * sc_hi * sc_lo, s1 = x1 * sc_hi * sc_lo;
    if (lane < m) ts[lane] = (T)s0;
    if (lane + 32 < m) ts[lane + 32] = (T)s1;
    r.a = __shfl_sync(FULL, s0, 0);
    r.t0 = (lane >= 1) ? s0 : 0.0;
    r.y = s1;
    return r;
}

template <typename T>
__device__ __forceinline__ void reflector_finish(int m, const ReflScale& r, T* v, T* tb)
{
    const int lane = threadIdx.x & 31;
    if (r.zero) {
        if (lane < m) v[lane] = (T)(lane == 0 ? 1.0 : 0.0);
        if (lane + 32 < m) v[lane + 32] = (T)0;
        if (lane == 0) { tb[0] = (T)0; tb[1] = (T)r.alpha; tb[2] = (T)0; }
        return;
    }
    const double a = r.a;
    double part = fma(r.t0, r.t0, r.y * r.y);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(FULL, part, o);
    const double s2 = fma(a, a, part);
    constexpr int NS = sizeof(T) == 8 ? 2 : 1;   // Newton steps for the storage precision
    const double rs = newton_rsqrt<NS>(s2);
    const double nrm = s2 * rs;
    const double absa = fabs(a);
    const double tau = fma(absa, rs, 1.0);
    const double rd = newton_rcp<NS>(absa + nrm);
    const double sgn = (r.alpha >= 0.0) ? 1.0 : -1.0;
    const double vs = sgn * rd;
    if (lane < m) v[lane] = (T)(lane == 0 ? 1.0 : r.t0 * vs);
    if (lane + 32 < m) v[lane + 32] = (T)(r.y * vs);
    if (lane == 0) {
        tb[0] = (T)tau;
        tb[1] = (T)((-sgn * nrm) * r.inv_hi * r.inv_lo);
        tb[2] = (T)vs;
    }
}

// Both halves in one call (used where nothing else overlaps).
template <typename T>
__device__ __forceinline__ void warp_reflector(int m, const T* x, T* ts, T* v, T* tb)
{
    const ReflScale r = reflector_scale<T>(m, x, ts);
    reflector_finish<T>(m, r, v, tb);
}

// ----------------------------------------------------------- bounded waits
// Spin until *addr >= target.  The sleep between polls grows with the
// distance still to go (a far-away target is polled rarely, so hundreds of
// waiting CTAs do not flood the L2 slice that holds the word).  Gives up (sets
// the error and abort words and returns false) when the watched word has not
// changed for timeout_ns, or when another CTA aborted.  Called by one thread.
// The polls are relaxed loads; one acquire load follows once the target is
// seen (the words only grow, so it reads a value >= target and synchronises
// with the release that wrote it).  An acquire at GPU scope also discards the
// SM's L1 contents, so polling with it would stall the other warps and CTAs
// of the SM on every poll.
__device__ bool wait_at_least(const int* addr, int target, Header* hdr,
                              unsigned long long timeout_ns)
{
    int last = ld_relaxed(addr);
    if (last >= target) { (void)ld_acquire(addr); return true; }
    unsigned long long t_last = global_ns();
    for (;;) {
        const int gap = target - last;
        __nanosleep(gap > 2 ? 2000u : (gap == 2 ? 400u : 64u));
        const int v = ld_relaxed(addr);
        if (v >= target) { (void)ld_acquire(addr); return true; }
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

}  // namespace bb

namespace bb {

// ---------------------------------------------- short-chain reflector (warp)
// FP64 approximations from the hardware's special-function unit (PTX
// rsqrt.approx / rcp.approx), refined below by published iterations.
__device__ __forceinline__ double rsqrt_approx(double x)
{
    double y;
    asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    return y;
}
__device__ __forceinline__ double rcp_approx(double x)
{
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    return y;
}

// Warp-cooperative Householder vector with the xLARFG contract (as
// warp_reflector), written for a short dependent chain: each dependent FP64
// operation costs about 63 cycles on this GPU, so the chain, not the
// arithmetic, sets the time of a reflector.
//   sum of squares  FP32 data: exact in 64-bit fixed point (each square is a
//                   48-bit integer; aligned to the largest exponent with 9
//                   bits of headroom for 33 terms, the truncation of small
//                   terms is below 2^-52 of the sum), one conversion to FP64;
//                   FP64 data: scaled by the power of two that brings the
//                   largest entry into [1, 4), squares summed in FP64.
//   norm            Goldschmidt's coupled iteration for sqrt(s) and
//                   1/(2 sqrt(s)) from the rsqrt.approx seed (STEPS steps).
//   1 / (|alpha| + norm)  Newton-Raphson from the rcp.approx seed.
// STEPS = 1 gives about 2^-44 (results rounded to FP32), 2 full FP64.
// x[0..m) in shared memory (m <= 64) -> v[0..MAXM) (zero beyond m),
// tb = {tau, beta, ...}; tau = 0 and v = e1 when x[1..m) is zero.
template <typename T, int MAXM>
__device__ __forceinline__ void fast_reflector(int m, const T* x, T* v, T* tb)
{
    const int lane = threadIdx.x & 31;
    constexpr int STEPS = sizeof(T) == 8 ? 2 : 1;
    const T x0 = lane < m ? x[lane] : (T)0;
    const T x1 = lane + 32 < m ? x[lane + 32] : (T)0;
    const T alpha = __shfl_sync(FULL, x0, 0);
    const bool zero = (m <= 1) || !__any_sync(FULL, (lane >= 1 && x0 != (T)0) || x1 != (T)0);
    if (zero) {
        for (int t = lane; t < MAXM; t += 32) v[t] = (T)(t == 0 ? 1 : 0);
        if (lane == 0) { tb[0] = (T)0; tb[1] = alpha; tb[2] = (T)0; }
        return;
    }
    double s2, inv_sc = 1.0;   // sum of squares of the (scaled) vector; 1 / scale
    double t0, t1;             // this lane's (scaled) entries in FP64
    if constexpr (sizeof(T) == 4) {
        // exact fixed-point sum of squares of FP32 values
        auto split = [](float f, unsigned& e, unsigned long long& q) {
            const unsigned u = __float_as_uint(f);
            e = (u >> 23) & 0xffu;
            unsigned mant = u & 0x7fffffu;
            if (e) mant |= 0x800000u; else e = 1;   // subnormal: exponent field 1
            q = (unsigned long long)mant * mant;     // < 2^48
            if (mant == 0) e = 0;
        };
        unsigned e0, e1;
        unsigned long long q0, q1;
        split((float)x0, e0, q0);
        split((float)x1, e1, q1);
        const unsigned E = __reduce_max_sync(FULL, max(e0, e1));
        const unsigned sh0 = 2 * (E - e0), sh1 = 2 * (E - e1);
        unsigned long long acc = (e0 && sh0 < 64 ? (q0 << 9) >> sh0 : 0ull) +
                                 (e1 && sh1 < 64 ? (q1 << 9) >> sh1 : 0ull);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
        // value = acc * 2^(2E - 300 - 9); split the power so each factor is normal
        const int p = 2 * (int)E - 309;
        const double f1 = __longlong_as_double((long long)(1023 + p / 2) << 52);
        const double f2 = __longlong_as_double((long long)(1023 + p - p / 2) << 52);
        s2 = ((double)acc * f1) * f2;
        t0 = (double)x0;
        t1 = (double)x1;
    } else {
        auto expo = [](double a) { return (unsigned)(__double_as_longlong(a) >> 52) & 0x7ffu; };
        const unsigned ef = __reduce_max_sync(FULL, max(expo(x0), expo(x1)));
        if (ef != 0) {
            const unsigned es = min(ef, 2045u);
            const double sc = __longlong_as_double((long long)(2046u - es) << 52);   // 2^(1023 - es)
            inv_sc = __longlong_as_double((long long)es << 52);                      // 2^(es - 1023)
            t0 = x0 * sc;
            t1 = x1 * sc;
        } else {   // every entry subnormal or zero
            t0 = (x0 * 0x1p1022) * 0x1p52;
            t1 = (x1 * 0x1p1022) * 0x1p52;
            inv_sc = 0x1p-1074;
        }
        double part = t0 * t0;
        if (m > 32) part = fma(t1, t1, part);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(FULL, part, o);
        s2 = part;
    }
    // Goldschmidt: g -> sqrt(s2), h -> 1 / (2 sqrt(s2))
    const double y = rsqrt_approx(s2);
    double g = s2 * y, h = 0.5 * y;
#pragma unroll
    for (int i = 0; i < STEPS; ++i) {
        const double r = fma(-g, h, 0.5);
        g = fma(g, r, g);
        h = fma(h, r, h);
    }
    const double a = __shfl_sync(FULL, t0, 0);
    const double absa = fabs(a);
    const double tau = fma(absa, h + h, 1.0);      // (beta - alpha) / beta = 1 + |alpha| / norm
    const double den = absa + g;
    double rd = rcp_approx(den);
#pragma unroll
    for (int i = 0; i < STEPS; ++i) {
        const double e = fma(-den, rd, 1.0);
        rd = fma(rd, e, rd);
    }
    // vs = sign(alpha) / (|alpha| + norm): the sign by the bit of alpha (sign(+-0) = +1)
    const bool neg = alpha < (T)0;
    const double vs = neg ? -rd : rd;
    if constexpr (sizeof(T) == 4) {
        if (fabs(vs) < 1e38) {        // vs fits FP32: one FP32 product per entry
            const float vsf = (float)vs;
            if (lane < MAXM) v[lane] = lane == 0 ? 1.0f : (lane < m ? (float)x0 * vsf : 0.0f);
            if (lane + 32 < MAXM) v[lane + 32] = lane + 32 < m ? (float)x1 * vsf : 0.0f;
        } else {                      // a vector of FP32 subnormals: the product in FP64
            if (lane < MAXM) v[lane] = lane == 0 ? 1.0f : (lane < m ? (float)(t0 * vs) : 0.0f);
            if (lane + 32 < MAXM) v[lane + 32] = lane + 32 < m ? (float)(t1 * vs) : 0.0f;
        }
    } else {
        if (lane < MAXM) v[lane] = lane == 0 ? 1.0 : (lane < m ? t0 * vs : 0.0);
        if (lane + 32 < MAXM) v[lane + 32] = lane + 32 < m ? t1 * vs : 0.0;
    }
    if (lane == 0) {
        tb[0] = (T)tau;
        tb[1] = (T)((neg ? g : -g) * inv_sc);
        tb[2] = (T)vs;
    }
}

}  // namespace bb
