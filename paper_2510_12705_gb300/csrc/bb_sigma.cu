// Singular values of the upper bidiagonal B = bidiag(d, e) on the GPU (the
// third SVD stage that the paper leaves to LAPACK, Sections V-A and VII).
//
// The Golub-Kahan matrix T_GK (order 2n, zero diagonal, off-diagonal
// f = (d0, e0, d1, e1, ..., d_{n-1})) has eigenvalues +-sigma_k.  For x > 0 its
// Sturm count (negative pivots of the LDL^T factorisation of T_GK - x I,
// q_0 = -x, q_i = -x - f_{i-1}^2 / q_{i-1}) equals n + #{sigma < x}.  Each
// thread finds one singular value by bisection on [0, ub], ub a Gershgorin
// bound, to the absolute accuracy eps * ub (relative accuracy for the values
// near the top), in FP64 whatever the storage type (the FP32 form's d, e are
// widened).
// The count runs the three-term Sturm recurrence: no divisions, exact
// power-of-two rescaling, restarts at splits, LAPACK's zero-pivot rule.
#include <cuda_runtime.h>

#include <algorithm>
#include <cfloat>
#include <cstdint>

#include "../../include/band_bidiag.h"

namespace {

constexpr unsigned FULL = 0xffffffffu;

// Bounds of the bisection, for the matrix scaled by the power of two sc that
// brings the largest |f_i| into [1, 2) (exact; without it f_i^2 overflows for
// entries above ~1e154): out = {ub, pivmin, sc, 1/sc} with
// ub = sc * max_i (|f_{i-1}| + |f_i|) and pivmin = (sc * max |f_i|)^2 * DBL_MIN.
// One block.
template <typename T>
__global__ void sigma_bounds_kernel(int64_t n, const T* __restrict__ d, const T* __restrict__ e,
                                    double* __restrict__ out)
{
    __shared__ double s_ub[32], s_fm[32];
    double ub = 0.0, fm = 0.0;
    const int64_t m = 2 * n - 1;   // number of off-diagonal entries of T_GK
    for (int64_t i = threadIdx.x; i < m; i += blockDim.x) {
        const double fi = (i & 1) ? (double)e[i >> 1] : (double)d[i >> 1];
        const double fp = (i == 0) ? 0.0 : ((i & 1) ? (double)d[i >> 1] : (double)e[(i >> 1) - 1]);
        ub = fmax(ub, 0.5 * fabs(fi) + 0.5 * fabs(fp));     // halved: no overflow near DBL_MAX
        fm = fmax(fm, fabs(fi));
    }
    for (int o = 16; o > 0; o >>= 1) {
        ub = fmax(ub, __shfl_xor_sync(FULL, ub, o));
        fm = fmax(fm, __shfl_xor_sync(FULL, fm, o));
    }
    if ((threadIdx.x & 31) == 0) { s_ub[threadIdx.x >> 5] = ub; s_fm[threadIdx.x >> 5] = fm; }
    __syncthreads();
    if (threadIdx.x < 32) {
        const int nw = blockDim.x >> 5;
        ub = (threadIdx.x < nw) ? s_ub[threadIdx.x] : 0.0;
        fm = (threadIdx.x < nw) ? s_fm[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) {
            ub = fmax(ub, __shfl_xor_sync(FULL, ub, o));
            fm = fmax(fm, __shfl_xor_sync(FULL, fm, o));
        }
        if (threadIdx.x == 0) {
            double sc = 1.0, isc = 1.0;
            if (fm > 0.0) {
                int ex = 0;
                frexp(fm, &ex);                                    // fm = f 2^ex, f in [0.5, 1)
                const int k = min(max(1 - ex, -1022), 1023);       // sc fm in [1, 2) unless subnormal
                sc = ldexp(1.0, k);
                isc = ldexp(1.0, -k);
            }
            const double fms = fm * sc;
            out[0] = 2.0 * (ub * sc) * (1.0 + 4.0 * DBL_EPSILON) + DBL_MIN;   // strictly above sigma_max
            out[1] = fmax(fms * fms * DBL_MIN, DBL_MIN);
            out[2] = sc;
            out[3] = isc;
        }
    }
}

// f2[i] = (sc f_i)^2, i < 2n - 1: the squared couplings of the scaled
// Golub-Kahan matrix, computed once for all the counts.
template <typename T>
__global__ void sigma_squares_kernel(int64_t n, const T* __restrict__ d, const T* __restrict__ e,
                                     const double* __restrict__ bounds, double* __restrict__ f2)
{
    const double sc = bounds[2];
    const int64_t m = 2 * n - 1;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double fi = ((i & 1) ? (double)e[i >> 1] : (double)d[i >> 1]) * sc;
        f2[i] = fi * fi;
    }
}

// #{sigma < x} for x > 0: the sign changes of the Sturm sequence p_0 = 1,
// p_1 = -x, p_i = -x p_{i-1} - f_{i-1}^2 p_{i-2} (the LDL^T pivots are
// q_i = p_i / p_{i-1}; a sign change is a negative pivot).  In this form a
// pivot costs one multiply and one FMA on the FP64 pipe and no division; the
// tests on zero and the exponent checks are integer operations on the bits.
//   - f_{i-1}^2 == 0 splits the matrix: the sequence restarts (q_i = -x < 0);
//   - an exactly zero p_i is replaced by -pivmin p_{i-1} (the pivot rule of
//     LAPACK's bisection; an underflow to a signed zero keeps the sign);
//   - the pair (p_{i-1}, p_i) is rescaled by an exact power of two after every
//     fourth pivot when its exponent leaves [-400, 400].  Bounds: in the
//     scaled matrix (max |f| in [1, 2)) a pivot grows the pair by less than 16;
//     it shrinks the pair by at most x unless the pivot cancels, and the
//     bisection never evaluates x below about 2^-55 ub (it stops at an absolute
//     accuracy of eps * sigma_max), so four pivots shrink it by at most about
//     2^-220 and the pair stays normal between checks.  A cancelling pivot is
//     followed by a large one.  (For x far below that range a run of tiny
//     couplings can underflow the pair; the count is used only on this range,
//     where tests/test_sigma_recurrence.py compares it with the oracle's.)
__device__ __forceinline__ void sturm_step(double& pm1, double& p, double f2, double mx, double pivmin,
                                           unsigned& neg)
{
    if (__double_as_longlong(f2) == 0) {        // f2 >= +0 always
        pm1 = 1.0;
        p = mx;
        neg += 1;
        return;
    }
    double pn = fma(mx, p, -(f2 * pm1));
    long long pb = __double_as_longlong(pn);
    if ((pb << 1) == 0) {                       // +-0
        pn = (__double_as_longlong(p) << 1) != 0 ? -pivmin * p : -pivmin;
        pb = __double_as_longlong(pn);
    }
    neg += (unsigned)((pb ^ __double_as_longlong(p)) < 0);   // sign change
    pm1 = p;
    p = pn;
}

__device__ __forceinline__ void sturm_rescale(double& pm1, double& p)
{
    const int e1 = (int)((__double_as_longlong(pm1) >> 52) & 0x7ff);
    const int e2 = (int)((__double_as_longlong(p) >> 52) & 0x7ff);
    const int ex = max(e1, e2) - 1023;          // exponent of max(|pm1|, |p|); -1023 for 0 / subnormal
    if (ex > 400 || ex < -400) {
        const double s = __longlong_as_double((long long)(1023 - ex) << 52);   // 2^-ex, finite
        pm1 *= s;
        p *= s;
    }
}

// #{sigma < x} from the squared couplings f2[0 .. 2n-2]
__device__ __forceinline__ unsigned count_below(int64_t n, const double* __restrict__ f2, double x,
                                                double pivmin)
{
    const double mx = -x;
    double pm1 = 1.0, p = mx;    // p_0, p_1
    if (fabs(p) < pivmin) p = -pivmin;
    unsigned neg = 1;            // p_0 > 0 > p_1
    const int64_t m = 2 * n - 1;
    int64_t i = 0;
    for (; i + 4 <= m; i += 4) {
        const double a0 = __ldg(f2 + i), a1 = __ldg(f2 + i + 1), a2 = __ldg(f2 + i + 2),
                     a3 = __ldg(f2 + i + 3);
        sturm_step(pm1, p, a0, mx, pivmin, neg);
        sturm_step(pm1, p, a1, mx, pivmin, neg);
        sturm_step(pm1, p, a2, mx, pivmin, neg);
        sturm_step(pm1, p, a3, mx, pivmin, neg);
        sturm_rescale(pm1, p);
    }
    for (; i < m; ++i) sturm_step(pm1, p, __ldg(f2 + i), mx, pivmin, neg);
    return neg - (unsigned)n;
}

// cnt[k] = #{sigma < ub k / G}, k = 1 .. G-1 (cnt[0] = 0, cnt[G] = n): a
// shared first cut of [0, ub] that replaces the first log2(G) halvings of
// every value's bisection
__global__ void sigma_grid_kernel(int64_t n, const double* __restrict__ f2, const double* __restrict__ bounds,
                                  int G, unsigned* __restrict__ cnt)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k > G) return;
    if (k == 0) { cnt[0] = 0; return; }
    if (k == G) { cnt[G] = (unsigned)n; return; }
    cnt[k] = count_below(n, f2, bounds[0] * ((double)k / (double)G), bounds[1]);
}

// thread j: the (j+1)-th smallest singular value, written to sigma[n-1-j]
// (descending order, like LAPACK's xBDSQR)
__global__ void sigma_bisect_kernel(int64_t n, const double* __restrict__ f2, const double* __restrict__ bounds,
                                    int G, const unsigned* __restrict__ cnt, double* __restrict__ sigma)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const double ub = bounds[0], pivmin = bounds[1], isc = bounds[3];
    // first cut: grid cell [ub k / G, ub (k+1) / G] with cnt[k] <= j < cnt[k+1]
    // (a search that keeps exactly that invariant, valid even if the computed
    // counts were not monotone)
    int klo = 0, khi = G;
    while (khi - klo > 1) {
        const int km = (klo + khi) >> 1;
        if ((int64_t)__ldg(cnt + km) <= j) klo = km; else khi = km;
    }
    double lo = klo == 0 ? 0.0 : ub * ((double)klo / (double)G);
    double hi = khi == G ? ub : ub * ((double)khi / (double)G);
    // invariant: #{sigma < lo} <= j < #{sigma < hi}.  Stop at the FP64
    // resolution around the value or at the absolute accuracy eps * ub (the
    // accuracy of any backward-stable bidiagonal SVD, and what bisection can
    // guarantee for values far below sigma_max): at most ~55 halvings in all
    const double abs_tol = 0.5 * DBL_EPSILON * ub;
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (hi - lo <= fmax(2.0 * DBL_EPSILON * fmax(fabs(lo), fabs(hi)), abs_tol) + 2.0 * pivmin) break;
        if ((int64_t)count_below(n, f2, mid, pivmin) > j) hi = mid; else lo = mid;
    }
    sigma[n - 1 - j] = (0.5 * (lo + hi)) * isc;
}

// grid size: a power of two, about half a count per singular value, at most 2^14
int grid_cells(int64_t n)
{
    int G = 1;
    while (G < 16384 && 4 * (int64_t)G <= n) G <<= 1;
    return G;
}

constexpr size_t kCntOffset = 256;
constexpr size_t kF2Offset = kCntOffset + 4 * (16384 + 1 + 63);   // 66048, 256-byte aligned

}  // namespace

extern "C" {

size_t bb_bidiag_sigma_workspace_size(int64_t n)
{
    // bounds (256 B) | grid counts | squared couplings (2n doubles)
    return kF2Offset + (size_t)(n > 0 ? n : 0) * 16;
}

int bb_bidiag_sigma(int64_t n, int dtype, const void* d, const void* e, double* sigma_out,
                    void* workspace, size_t ws_bytes, void* stream)
{
    if (n < 1 || (dtype != BB_F32 && dtype != BB_F64) || !d || (n > 1 && !e) || !sigma_out)
        return BB_ERR_ARG;
    if (n >= ((int64_t)1 << 31)) return BB_ERR_UNSUPPORTED;
    if (!workspace || ws_bytes < bb_bidiag_sigma_workspace_size(n) || ((uintptr_t)workspace & 15))
        return BB_ERR_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned char* ws = (unsigned char*)workspace;
    double* bounds = (double*)ws;
    unsigned* cnt = (unsigned*)(ws + kCntOffset);
    double* f2 = (double*)(ws + kF2Offset);
    const int G = grid_cells(n);
    const unsigned sq_grid = (unsigned)std::min<int64_t>((2 * n - 1 + 255) / 256, 1184);
    if (dtype == BB_F64) {
        sigma_bounds_kernel<double><<<1, 1024, 0, st>>>(n, (const double*)d, (const double*)e, bounds);
        sigma_squares_kernel<double><<<sq_grid, 256, 0, st>>>(n, (const double*)d, (const double*)e, bounds, f2);
    } else {
        sigma_bounds_kernel<float><<<1, 1024, 0, st>>>(n, (const float*)d, (const float*)e, bounds);
        sigma_squares_kernel<float><<<sq_grid, 256, 0, st>>>(n, (const float*)d, (const float*)e, bounds, f2);
    }
    // one warp per block: each thread is a long dependent FP64 chain, so
    // spreading the work over all SMs beats packing warps onto a few
    sigma_grid_kernel<<<(unsigned)((G + 1 + 31) / 32), 32, 0, st>>>(n, f2, bounds, G, cnt);
    sigma_bisect_kernel<<<(unsigned)((n + 31) / 32), 32, 0, st>>>(n, f2, bounds, G, cnt, sigma_out);
    return cudaGetLastError() == cudaSuccess ? BB_OK : BB_ERR_LAUNCH;
}

}  // extern "C"
