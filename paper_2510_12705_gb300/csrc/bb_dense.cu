// Stage 1 of the SVD on the GPU: a dense n x n matrix to upper band form with
// bandwidth b (arXiv 2510.12705, Section II: the two-stage approach reduces the
// dense matrix to a band first; Section V-A: the accuracy experiments start
// from dense matrices with prescribed singular values).
//
// B = Q^T A P by Householder reflectors, one b-wide panel at a time:
//   column panel k: Householder QR of columns k .. k+w-1 (rows k .. n-1), then
//     the compact-WY update A2 <- A2 - V (T^T (V^T A2)) of the columns to its
//     right (w = min(b, n - k));
//   row panel k: Householder LQ of rows k .. k+w-1 beyond the diagonal block,
//     done as the QR of the transposed row panel, then the update
//     A3 <- A3 - ((A3 U) T) U^T of the rows below it.
// The panel factorisations are this file's kernels (one CTA per panel: block
// reductions for the norms, a warp per column for the updates, the LAPACK
// larfg convention); T comes from the Gram matrix V^T V by the forward
// recurrence T[j][j] = tau_j, T[0:j][j] = -tau_j T[0:j][0:j] (V^T v_j); the
// trailing updates are plain GEMMs (cuBLAS).  Every reflector is the one the
// unblocked algorithm computes: blocking only groups their application to
// the trailing matrix.
#include <cublas_v2.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <mutex>
#include <vector>

#include "../../include/band_bidiag.h"

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int PANEL_THREADS = 1024;

// block-wide sum / max over PANEL_THREADS threads (shared scratch of 32)
template <typename T>
__device__ __forceinline__ T block_sum(T v, T* red)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    v = lane < (int)(blockDim.x >> 5) ? red[lane] : (T)0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}
template <typename T>
__device__ __forceinline__ T block_max(T v, T* red)
{
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(FULL, v, o));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    v = lane < (int)(blockDim.x >> 5) ? red[lane] : (T)0;
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(FULL, v, o));
    return v;
}

// Householder QR of the m x wc panel X (column-major, leading dimension ldx)
// with nrefl = min(m, wc) reflectors, one CTA.  Reflector j comes from column
// j, rows j .. m-1 (larfg: beta = -sign(alpha) ||x||, sign(0) = +1, tau = 0 for
// a zero tail), is applied to columns j+1 .. wc-1, and leaves (beta, 0..0) in
// X; its vector (unit first entry, zeros above) goes to column j of V (ldv),
// tau to tau[j].  The norm is scaled by the tail's largest magnitude, so its
// square cannot overflow or underflow.  The arithmetic is in T (FP32 or FP64).
template <typename T>
__global__ void __launch_bounds__(PANEL_THREADS) panel_qr_kernel(T* __restrict__ X, int64_t ldx, int m, int wc,
                                                                 int nrefl, T* __restrict__ V, int64_t ldv,
                                                                 T* __restrict__ tau)
{
    __shared__ T red[32];
    __shared__ T s_tau, s_scal;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    for (int j = 0; j < nrefl; ++j) {
        T* x = X + (int64_t)j * ldx;
        // largest magnitude of the tail x[j+1 .. m-1]
        T amax = (T)0;
        for (int i = j + 1 + tid; i < m; i += nt) amax = max(amax, fabs(x[i]));
        amax = block_max(amax, red);
        if (amax == (T)0) {
            // H = I: nothing to apply; v = e_j
            for (int i = tid; i < m; i += nt) V[i + (int64_t)j * ldv] = (T)(i == j ? 1 : 0);
            if (tid == 0) tau[j] = (T)0;
            __syncthreads();
            continue;
        }
        const T inv = (T)1 / amax;
        T ss = (T)0;
        for (int i = j + 1 + tid; i < m; i += nt) {
            const T t = x[i] * inv;
            ss = fma(t, t, ss);
        }
        ss = block_sum(ss, red);
        if (tid == 0) {
            const T alpha = x[j];
            const T xnorm = amax * sqrt(ss);
            const T beta = -copysign(hypot(alpha, xnorm), alpha != (T)0 ? alpha : (T)1);
            s_tau = (beta - alpha) / beta;
            s_scal = (T)1 / (alpha - beta);
            tau[j] = s_tau;
            x[j] = beta;
        }
        __syncthreads();
        const T scal = s_scal, tj = s_tau;
        for (int i = tid; i < m; i += nt) {
            T vi;
            if (i < j) vi = (T)0;
            else if (i == j) vi = (T)1;
            else {
                vi = x[i] * scal;
                x[i] = vi;          // the lower part of X keeps v (outside the band)
            }
            V[i + (int64_t)j * ldv] = vi;
        }
        __syncthreads();
        // apply H_j = I - tau v v^T to columns j+1 .. wc-1: a warp per column
        for (int cc = j + 1 + warp; cc < wc; cc += nw) {
            T* y = X + (int64_t)cc * ldx;
            const T* v = V + (int64_t)j * ldv;
            T d0 = (T)0, d1 = (T)0, d2 = (T)0, d3 = (T)0;   // four chains for the FP64 latency
            int i = j + lane;
            for (; i + 96 < m; i += 128) {
                d0 = fma(v[i], y[i], d0);
                d1 = fma(v[i + 32], y[i + 32], d1);
                d2 = fma(v[i + 64], y[i + 64], d2);
                d3 = fma(v[i + 96], y[i + 96], d3);
            }
            for (; i < m; i += 32) d0 = fma(v[i], y[i], d0);
            T d = (d0 + d1) + (d2 + d3);
            for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(FULL, d, o);
            const T f = tj * d;
            for (int i = j + lane; i < m; i += 32) y[i] = fma(-f, v[i], y[i]);
        }
        __syncthreads();
    }
}

// T factor (w x w, upper triangular, leading dimension ldt) of the forward
// product H_0 H_1 ... H_{w-1} = I - V T V^T from the Gram matrix G = V^T V
// (ldg) and tau: T[j][j] = tau_j, T[0:j][j] = -tau_j T[0:j][0:j] G[0:j][j].
// One CTA; the rows i < j of column j are independent.
template <typename T>
__global__ void build_t_kernel(const T* __restrict__ G, int64_t ldg, const T* __restrict__ tau, int w,
                               T* __restrict__ Tm, int64_t ldt)
{
    for (int idx = threadIdx.x; idx < w * w; idx += blockDim.x) Tm[(idx % w) + (int64_t)(idx / w) * ldt] = (T)0;
    __syncthreads();
    for (int j = 0; j < w; ++j) {
        const T tj = tau[j];
        for (int i = threadIdx.x; i <= j; i += blockDim.x) {
            if (i == j) {
                Tm[i + (int64_t)j * ldt] = tj;
            } else {
                T s = (T)0;
                for (int l = i; l < j; ++l) s = fma(Tm[i + (int64_t)l * ldt], G[l + (int64_t)j * ldg], s);
                Tm[i + (int64_t)j * ldt] = -tj * s;
            }
        }
        __syncthreads();
    }
}

// dst (rows x cols, leading dimension ldd) = the transpose of src (cols x
// rows, lds): dst[r + c ldd] = src[c + r lds]; with `upper_zero`, entries with
// c > r are written as exact zeros.  32 x 32 tiles through shared memory, both
// sides coalesced.
template <typename T>
__global__ void transpose_kernel(const T* __restrict__ src, int64_t lds, T* __restrict__ dst, int64_t ldd,
                                 int rows, int cols, int upper_zero)
{
    __shared__ T tile[32][33];
    const int bx = blockIdx.x * 32, by = blockIdx.y * 32;   // dst rows, dst columns
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int r = bx + k, c = by + threadIdx.x;
        if (r < rows && c < cols) tile[k][threadIdx.x] = src[c + (int64_t)r * lds];
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int r = bx + threadIdx.x, c = by + k;
        if (r < rows && c < cols) dst[r + (int64_t)c * ldd] = (upper_zero && c > r) ? (T)0 : tile[threadIdx.x][k];
    }
}

// band_out[(b + i - j) + j ldab] = A[i + j lda] for 0 <= j - i <= b (slots
// above row 0 set to zero)
template <typename T>
__global__ void extract_band_kernel(const T* __restrict__ A, int64_t lda, int n, int b, T* __restrict__ band,
                                    int64_t ldab)
{
    const int64_t total = (int64_t)n * (b + 1);
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(t / (b + 1)), k = (int)(t % (b + 1));   // k = b + i - j
        const int i = j - b + k;
        band[k + (int64_t)j * ldab] = i >= 0 ? A[i + (int64_t)j * lda] : (T)0;
    }
}

template <typename T>
__global__ void copy_matrix_kernel(const T* __restrict__ src, int64_t lds, T* __restrict__ dst, int64_t ldd, int n)
{
    const int64_t total = (int64_t)n * n;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(t / n), i = (int)(t % n);
        dst[i + (int64_t)j * ldd] = src[i + (int64_t)j * lds];
    }
}

// ------------------------------------------------------------------ host

constexpr size_t kAlign = 256;
inline size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

struct DenseLayout {
    size_t a, v, p, t, g, w1, w2, tau, bytes;
};

DenseLayout dense_layout(int64_t n, int64_t b, size_t es)
{
    DenseLayout L{};
    size_t off = 0;
    const size_t nn = (size_t)n, bb = (size_t)std::max<int64_t>(b, 1);
    L.a = off;   off = align_up(off + es * nn * nn);        // working copy of A (ld n)
    L.v = off;   off = align_up(off + es * nn * bb);        // panel reflectors (ld n)
    L.p = off;   off = align_up(off + es * nn * bb);        // transposed row panel (ld n)
    L.t = off;   off = align_up(off + es * bb * bb);        // T factor (ld b)
    L.g = off;   off = align_up(off + es * bb * bb);        // Gram matrix (ld b)
    L.w1 = off;  off = align_up(off + es * nn * bb);        // GEMM products (ld n or b)
    L.w2 = off;  off = align_up(off + es * nn * bb);
    L.tau = off; off = align_up(off + es * bb);
    L.bytes = off;
    return L;
}

// one cuBLAS handle per device, created on first use; calls on a device
// serialise on its mutex (the handle's stream is set per call)
std::mutex g_blas_mu;
std::vector<cublasHandle_t> g_blas;

cublasHandle_t blas_handle(int dev)
{
    if ((int)g_blas.size() <= dev) g_blas.resize(dev + 1, nullptr);
    if (!g_blas[dev] && cublasCreate(&g_blas[dev]) != CUBLAS_STATUS_SUCCESS) g_blas[dev] = nullptr;
    return g_blas[dev];
}

cublasStatus_t gemm(cublasHandle_t h, cublasOperation_t ta, cublasOperation_t tb, int m, int n, int k, double alpha,
                    const double* A, int64_t lda, const double* B, int64_t ldb, double beta, double* C, int64_t ldc)
{
    return cublasDgemm(h, ta, tb, m, n, k, &alpha, A, (int)lda, B, (int)ldb, &beta, C, (int)ldc);
}
cublasStatus_t gemm(cublasHandle_t h, cublasOperation_t ta, cublasOperation_t tb, int m, int n, int k, float alpha,
                    const float* A, int64_t lda, const float* B, int64_t ldb, float beta, float* C, int64_t ldc)
{
    return cublasSgemm(h, ta, tb, m, n, k, &alpha, A, (int)lda, B, (int)ldb, &beta, C, (int)ldc);
}

template <typename T>
__global__ void set_identity_kernel(T* __restrict__ X, int64_t ldx, int n)
{
    const int64_t total = (int64_t)n * n;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(t / n), i = (int)(t % n);
        X[i + (int64_t)j * ldx] = (T)(i == j ? 1 : 0);
    }
}

// The reduction; with Qo / Po (n x n, column-major) also the orthogonal
// factors with Qo^T A Po = B: each panel's block of reflectors, I - V T V^T,
// multiplies them from the right (Qo: the column panel's, on its columns
// k .. n-1; Po: the row panel's, on its columns k+w .. n-1), in panel order.
template <typename T>
int dense_run(int64_t n64, int b, const T* A, int64_t lda, T* band, int64_t ldab, int64_t b_out, char* ws,
              cudaStream_t st, T* Qo = nullptr, int64_t ldq = 0, T* Po = nullptr, int64_t ldp = 0)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return BB_ERR_LAUNCH;
    std::lock_guard<std::mutex> lk(g_blas_mu);
    cublasHandle_t h = blas_handle(dev);
    if (!h || cublasSetStream(h, st) != CUBLAS_STATUS_SUCCESS ||
        cublasSetMathMode(h, CUBLAS_DEFAULT_MATH) != CUBLAS_STATUS_SUCCESS)
        return BB_ERR_LAUNCH;
    const int n = (int)n64;
    const DenseLayout Lo = dense_layout(n64, b, sizeof(T));
    T* Aw = (T*)(ws + Lo.a);
    T* V = (T*)(ws + Lo.v);
    T* P = (T*)(ws + Lo.p);
    T* Tm = (T*)(ws + Lo.t);
    T* G = (T*)(ws + Lo.g);
    T* W1 = (T*)(ws + Lo.w1);
    T* W2 = (T*)(ws + Lo.w2);
    T* tau = (T*)(ws + Lo.tau);
    const cublasOperation_t OT = CUBLAS_OP_T, ON = CUBLAS_OP_N;
    const int grid1 = (int)std::min<int64_t>(((int64_t)n * n + 255) / 256, 152 * 16);
    copy_matrix_kernel<T><<<grid1, 256, 0, st>>>(A, lda, Aw, n, n);
    bool ok = cudaGetLastError() == cudaSuccess;
    if (Qo) {
        set_identity_kernel<T><<<grid1, 256, 0, st>>>(Qo, ldq, n);
        set_identity_kernel<T><<<grid1, 256, 0, st>>>(Po, ldp, n);
        ok = ok && cudaGetLastError() == cudaSuccess;
    }
    const dim3 tb(32, 8);
    for (int k = 0; ok && k < n; k += b) {
        const int m = n - k, w = std::min(b, m), n2 = n - k - w;
        panel_qr_kernel<T><<<1, PANEL_THREADS, 0, st>>>(Aw + k + (int64_t)k * n, n, m, w, w, V, n, tau);
        ok = cudaGetLastError() == cudaSuccess;
        if (!ok || (n2 <= 0 && !Qo)) break;
        ok = gemm(h, OT, ON, w, w, m, (T)1, V, n, V, n, (T)0, G, b) == CUBLAS_STATUS_SUCCESS;
        build_t_kernel<T><<<1, std::min(1024, (w + 31) / 32 * 32), 0, st>>>(G, b, tau, w, Tm, b);
        ok = ok && cudaGetLastError() == cudaSuccess;
        if (Qo) {   // Qo[:, k:] <- Qo[:, k:] - ((Qo[:, k:] V) T) V^T
            T* Qc = Qo + (int64_t)k * ldq;
            ok = ok && gemm(h, ON, ON, n, w, m, (T)1, Qc, ldq, V, n, (T)0, W1, n) == CUBLAS_STATUS_SUCCESS;
            ok = ok && gemm(h, ON, ON, n, w, w, (T)1, W1, n, Tm, b, (T)0, W2, n) == CUBLAS_STATUS_SUCCESS;
            ok = ok && gemm(h, ON, OT, n, m, w, (T)-1, W2, n, V, n, (T)1, Qc, ldq) == CUBLAS_STATUS_SUCCESS;
        }
        if (!ok || n2 <= 0) break;
        // columns to the right: A2 <- A2 - V (T^T (V^T A2))
        T* A2 = Aw + k + (int64_t)(k + w) * n;
        ok = ok && gemm(h, OT, ON, w, n2, m, (T)1, V, n, A2, n, (T)0, W1, b) == CUBLAS_STATUS_SUCCESS;
        ok = ok && gemm(h, OT, ON, w, n2, w, (T)1, Tm, b, W1, b, (T)0, W2, b) == CUBLAS_STATUS_SUCCESS;
        ok = ok && gemm(h, ON, ON, m, n2, w, (T)-1, V, n, W2, b, (T)1, A2, n) == CUBLAS_STATUS_SUCCESS;
        if (!ok) break;
        // row panel (rows k .. k+w-1, columns k+w .. n-1) as the QR of its transpose
        const int w2 = std::min(w, n2);
        transpose_kernel<T><<<dim3((n2 + 31) / 32, (w + 31) / 32), tb, 0, st>>>(A2, n, P, n, n2, w, 0);
        panel_qr_kernel<T><<<1, PANEL_THREADS, 0, st>>>(P, n, n2, w, w2, V, n, tau);
        transpose_kernel<T><<<dim3((w + 31) / 32, (n2 + 31) / 32), tb, 0, st>>>(P, n, A2, n, w, n2, 1);
        ok = cudaGetLastError() == cudaSuccess;
        // rows below: A3 <- A3 - ((A3 U) T) U^T
        T* A3 = Aw + (k + w) + (int64_t)(k + w) * n;
        ok = ok && gemm(h, OT, ON, w2, w2, n2, (T)1, V, n, V, n, (T)0, G, b) == CUBLAS_STATUS_SUCCESS;
        build_t_kernel<T><<<1, std::min(1024, (w2 + 31) / 32 * 32), 0, st>>>(G, b, tau, w2, Tm, b);
        ok = ok && cudaGetLastError() == cudaSuccess;
        ok = ok && gemm(h, ON, ON, n2, w2, n2, (T)1, A3, n, V, n, (T)0, W1, n) == CUBLAS_STATUS_SUCCESS;
        ok = ok && gemm(h, ON, ON, n2, w2, w2, (T)1, W1, n, Tm, b, (T)0, W2, n) == CUBLAS_STATUS_SUCCESS;
        ok = ok && gemm(h, ON, OT, n2, n2, w2, (T)-1, W2, n, V, n, (T)1, A3, n) == CUBLAS_STATUS_SUCCESS;
        if (Po) {   // Po[:, k+w:] <- Po[:, k+w:] - ((Po[:, k+w:] U) T) U^T
            T* Pc = Po + (int64_t)(k + w) * ldp;
            ok = ok && gemm(h, ON, ON, n, w2, n2, (T)1, Pc, ldp, V, n, (T)0, W1, n) == CUBLAS_STATUS_SUCCESS;
            ok = ok && gemm(h, ON, ON, n, w2, w2, (T)1, W1, n, Tm, b, (T)0, W2, n) == CUBLAS_STATUS_SUCCESS;
            ok = ok && gemm(h, ON, OT, n, n2, w2, (T)-1, W2, n, V, n, (T)1, Pc, ldp) == CUBLAS_STATUS_SUCCESS;
        }
    }
    if (!ok) return BB_ERR_LAUNCH;
    const int grid2 = (int)std::min<int64_t>(((int64_t)n * (b_out + 1) + 255) / 256, 152 * 16);
    extract_band_kernel<T><<<grid2, 256, 0, st>>>(Aw, n, n, (int)b_out, band, ldab);
    return cudaGetLastError() == cudaSuccess ? BB_OK : BB_ERR_LAUNCH;
}

}  // namespace

extern "C" {

size_t dense_to_band_workspace_size(int64_t n, int64_t b, int dtype)
{
    if (n < 1 || b < 1 || (dtype != BB_F32 && dtype != BB_F64)) return 0;
    const int64_t bi = std::min<int64_t>(b, n);
    return dense_layout(n, bi, dtype == BB_F64 ? 8 : 4).bytes;
}

int dense_to_band(int64_t n, int64_t b, int dtype, const void* a, int64_t lda, void* band_out, int64_t ldab,
                  void* workspace, size_t ws_bytes, void* stream_ptr)
{
    cudaStream_t stream = (cudaStream_t)stream_ptr;
    if (n < 1 || b < 1 || lda < n || ldab < b + 1 || !a || !band_out) return BB_ERR_ARG;
    if (dtype != BB_F32 && dtype != BB_F64) return dtype == BB_F16 || dtype == BB_BF16 ? BB_ERR_UNSUPPORTED : BB_ERR_ARG;
    if (n > (int64_t)1 << 30) return BB_ERR_UNSUPPORTED;
    const int bi = (int)std::min<int64_t>(b, n);
    const size_t need = dense_to_band_workspace_size(n, b, dtype);
    void* ws = workspace;
    bool own = false;
    if (ws) {
        if (ws_bytes < need) return BB_ERR_WORKSPACE;
    } else {
        if (cudaMallocAsync(&ws, need, stream) != cudaSuccess) { cudaGetLastError(); return BB_ERR_ALLOC; }
        own = true;
    }
    const int rc = dtype == BB_F64
        ? dense_run<double>(n, bi, (const double*)a, lda, (double*)band_out, ldab, b, (char*)ws, stream)
        : dense_run<float>(n, bi, (const float*)a, lda, (float*)band_out, ldab, b, (char*)ws, stream);
    if (own && cudaFreeAsync(ws, stream) != cudaSuccess && rc == BB_OK) return BB_ERR_LAUNCH;
    return rc;
}

int dense_to_band_qp(int64_t n, int64_t b, int dtype, const void* a, int64_t lda, void* band_out, int64_t ldab,
                     void* q_out, int64_t ldq, void* p_out, int64_t ldp, void* workspace, size_t ws_bytes,
                     void* stream_ptr)
{
    cudaStream_t stream = (cudaStream_t)stream_ptr;
    if (n < 1 || b < 1 || lda < n || ldab < b + 1 || !a || !band_out || !q_out || !p_out || ldq < n || ldp < n)
        return BB_ERR_ARG;
    if (dtype != BB_F32 && dtype != BB_F64) return dtype == BB_F16 || dtype == BB_BF16 ? BB_ERR_UNSUPPORTED : BB_ERR_ARG;
    if (n > (int64_t)1 << 30) return BB_ERR_UNSUPPORTED;
    if (ldq > INT32_MAX || ldp > INT32_MAX) return BB_ERR_UNSUPPORTED;   // cuBLAS takes 32-bit leading dimensions
    const int bi = (int)std::min<int64_t>(b, n);
    const size_t need = dense_to_band_workspace_size(n, b, dtype);
    void* ws = workspace;
    bool own = false;
    if (ws) {
        if (ws_bytes < need) return BB_ERR_WORKSPACE;
    } else {
        if (cudaMallocAsync(&ws, need, stream) != cudaSuccess) { cudaGetLastError(); return BB_ERR_ALLOC; }
        own = true;
    }
    const int rc = dtype == BB_F64
        ? dense_run<double>(n, bi, (const double*)a, lda, (double*)band_out, ldab, b, (char*)ws, stream,
                            (double*)q_out, ldq, (double*)p_out, ldp)
        : dense_run<float>(n, bi, (const float*)a, lda, (float*)band_out, ldab, b, (char*)ws, stream,
                           (float*)q_out, ldq, (float*)p_out, ldp);
    if (own && cudaFreeAsync(ws, stream) != cudaSuccess && rc == BB_OK) return BB_ERR_LAUNCH;
    return rc;
}

}  // extern "C"
