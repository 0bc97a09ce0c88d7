// Device kernels of the factorization and the solve, templated on the storage
// type T of the factor (double for the FP64 path, float for the mixed path).
// Diagonal-tile Cholesky always computes in FP64.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace rsc {

constexpr int TILE = 64;      // output tile edge of the GEMM-shaped kernels
constexpr int KCH = 16;       // K chunk staged in shared memory
constexpr int NB = 64;        // panel width of the blocked tall-panel Cholesky
constexpr int SOLVE_MAX = 256;  // largest dense diagonal block solved inside one CTA

// ------------------------------------------------------------------ task records
struct PotrfTask { void* a; int ld; int nb; int node; };
struct TrsmTask { const void* L; void* B; int ldl; int ldb; int nb; int nrows; };
struct GemmTask {            // C[i,j] -= sum_l A[i,l] B[j,l]; lower mask i + moff >= j
    const void* A; const void* B; void* C;
    int lda, ldb, ldc, m, n, K, moff, lower;
};
struct PushTask { int k, j, pr0, pr1, pc0, pc1; };
struct LoOp { const void* base; int ld; int K; };   // rows of L^O_k or V_k
struct NodeTgt {             // where extend-add updates of supernode j go
    void* base;              // panel (kind 0) or dense diagonal (kind 1)
    int ld; int kind;        // 0 panel, 1 dense diagonal, 2 hierarchical leaves, 3 none
    int c; int r; long long c0; long long rows_off;
};
struct LeafMap { long long lo; long long off; int size; int pad; };   // per column of a hierarchical node
struct TnTask {              // Z[t, :] = beta Z[t, :] + alpha sum_i A[arow_i, t] Y[yrow_i, :]  (N columns)
    const void* A; int lda; int K; int nrow;
    const int32_t* amap; int aoff; const int32_t* ymap; int yoff;
    void* Z; int ldz; int t0;          // t0: first column of A of this CTA (8 columns, one per warp)
    const void* Y; int ldy; int N;
    double alpha, beta;
    // row split (k_tn only): CTA z of the task sums rows [z rps, (z + 1) rps) into
    // part[z][32][N]; the last CTA to arrive (counter cnt[chunk]) adds the nsplit partial
    // sums in ascending z and writes Z, then resets its counter.
    int nsplit = 1, rps = 0;
    void* part = nullptr;
    unsigned* cnt = nullptr;
};
struct NnTask {              // Y[yrow_i, :] += alpha sum_l A[arow_i, l] Z[l, :]  (N columns)
    const void* A; int lda; int K; int nrow;
    const int32_t* amap; int aoff; const int32_t* ymap; int yoff;
    const void* Z; int ldz; int row0;  // row0: first row of this CTA's 64-row chunk
    void* Y; int ldy; int N;
    double alpha; int atomic;
};
struct TrsvTask { const void* L; int ld; int c; int N; void* X; int ldx; int transpose; };
struct CsrBlock { const int32_t* rp; const int32_t* ci; const double* v; int nrows; int pad; };
// Y(row i, column c) = alpha (A X)(i, c), or added (mode 1; mode 2 atomically).  With rmap the
// output row of CSR row i is rmap[i]; with cmap column c goes to column cmap[c]; lower: only
// entries whose output column index is >= the output row index (the lower triangle of a
// column-major target written as rows of its transpose) are written.
struct CsrTask { CsrBlock blk; const void* X; int ldx; void* Y; int ldy; int N; int row0; double alpha;
                 const int32_t* rmap; const int32_t* cmap; int mode; int lower; };
struct GaussTask { void* G; int m; int row0; uint32_t block_id; uint32_t word3; int ld; int col0; };
struct CopyTask { const void* src; long long ssr, ssc; void* dst; long long dsr, dsc; int m, nc; int sub; };  // sub: dst -= src
// One action of a hierarchical (or blocked dense) diagonal solve, rows local to the block:
//   HA_TRSV   X[o0:o0+no] <- L^{-1} X[..] or L^{-T} X[..]   (A1 = row-major L^{-1}, no <= SOLVE_MAX)
//   HA_LR     X[o0:o0+no] -= A2 (A1^T X[i0:i0+ni])          (A1 ni x K, A2 no x K; low rank)
//   HA_GEMV   X[o0:o0+no] -= A2 X[i0:i0+K]                  (A2 no x K)
//   HA_GEMVT  X[o0:o0+no] -= A1^T X[i0:i0+ni]               (A1 ni x no)
enum { HA_TRSV = 0, HA_LR = 1, HA_GEMV = 2, HA_GEMVT = 3 };
struct HAct { int type, i0, ni, o0, no, K; const void* A1; int lda1; const void* A2; int lda2; };
struct HTask { const HAct* acts; long long nact; void* X; int ldx; int N; int c; int transpose; };

// ------------------------------------------------------------------ helpers
template <class T> __device__ __forceinline__ void atomic_add(T* p, T v) { atomicAdd(p, v); }

__device__ __forceinline__ int lower_bound_i32(const int32_t* a, int n, int32_t x) {
    int lo = 0, hi = n;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (a[mid] < x) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// ------------------------------------------------------------------ assembly
// arena[dst[e]] = val[src[e]] : A's lower triangle into the dense factor storage.
template <class T>
__global__ void k_assemble(const double* __restrict__ val, const long long* __restrict__ src,
                           const long long* __restrict__ dst, long long cnt, T* __restrict__ arena) {
    long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    long long stride = (long long)gridDim.x * blockDim.x;
    for (; e < cnt; e += stride) arena[dst[e]] = (T)val[src[e]];
}

// ------------------------------------------------------------------ diagonal tile Cholesky
// The tiles are factored in the storage precision: FP64 in the FP64 form; FP32 where the factor
// is stored in FP32 (on this part a warp's FP64 instruction holds its sub-partition about 64
// cycles, so the pivots' dependent chains dominated the hierarchical leaves; FP32's tile error,
// about 1e-7 relative, is far below the compression tolerances).
template <class T> struct TileType { using type = T; };
// 1 / sqrt(x) in FP32: the hardware estimate and one Newton step.
__device__ __forceinline__ float rsqrt_f32(float x) {
    const float y = rsqrtf(x);
    return y * fmaf(-0.5f * x * y, y, 1.5f);
}
// 1 / sqrt(x) by Newton's method for f(y) = y^-2 - x (y <- y (3 - x y^2) / 2), two steps from
// the single-precision estimate (about 22 correct bits -> 44 -> full double precision, within
// a few ulp).  On this part a dependent FP64 operation takes about 64 cycles, the library's
// FP64 square root about 690 and division about 440, so the pivot's square root and
// reciprocal come from these six operations.  Outside the float range the library is used.
// (The FP64 form uses two steps; the FP32-storage forms factor their tiles in FP32.)
template <int STEPS = 2>
__device__ __forceinline__ double rsqrt_newton(double x) {
    if (!(x > 1e-30 && x < 1e30)) return 1.0 / sqrt(x);
    double y = (double)rsqrtf((float)x);
    const double hx = 0.5 * x;
#pragma unroll
    for (int i = 0; i < STEPS; ++i) y = y * fma(-hx * y, y, 1.5);
    return y;
}

__device__ __forceinline__ double rsqrt_tile(double x) { return rsqrt_newton<2>(x); }
__device__ __forceinline__ float rsqrt_tile(float x) { return rsqrt_f32(x); }

// Cholesky of one nb x nb (nb <= 64) diagonal tile in the storage precision, lower triangle in
// place, in shared memory (right-looking).  Thread 0 forms the pivot's square root and
// reciprocal (rsqrt_tile); the column is scaled by multiplication, and the trailing update runs
// warps over columns, lanes down the rows of each column's lower part (no index division).
template <class T>
__global__ void __launch_bounds__(256) k_potrf_tile(const PotrfTask* __restrict__ tasks, int* status) {
    using TT = typename TileType<T>::type;
    __shared__ TT s[NB][NB + 1];
    __shared__ TT rpiv;
    const PotrfTask tk = tasks[blockIdx.x];
    T* a = (T*)tk.a;
    const int nb = tk.nb, ld = tk.ld;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int j = warp; j < nb; j += 8)
        for (int i = j + lane; i < nb; i += 32) s[i][j] = (TT)a[i + (size_t)j * ld];
    __syncthreads();
    for (int k = 0; k < nb; ++k) {
        if (threadIdx.x == 0) {
            TT d = s[k][k];
            if (!(d > TT(0))) {          // indefinite or NaN pivot: record, keep values finite
                atomicCAS(status, 0, tk.node + 1);
                d = TT(1);
            }
            const TT y = rsqrt_tile(d);
            s[k][k] = d * y;
            rpiv = y;
        }
        __syncthreads();
        const TT ri = rpiv;
        for (int i = k + 1 + threadIdx.x; i < nb; i += blockDim.x) s[i][k] *= ri;
        __syncthreads();
        for (int j = k + 1 + warp; j < nb; j += 8) {
            const TT ljk = s[j][k];
            for (int i = j + lane; i < nb; i += 32) s[i][j] = fma(-s[i][k], ljk, s[i][j]);
        }
        __syncthreads();
    }
    for (int j = warp; j < nb; j += 8)
        for (int i = j + lane; i < nb; i += 32) a[i + (size_t)j * ld] = (T)s[i][j];
}

// ------------------------------------------------------------------ whole leaf block in one CTA
// Cholesky of one sz x sz diagonal leaf (Alg. 6's leaf blocks, sz <= LEAF_FUSED_MAX) held in
// shared memory, by 32-column panels:
//  * the 32 x 32 diagonal tile in the storage precision by four warps, one per SM sub-partition:
//    per pivot every lane forms 1/sqrt by rsqrt_tile, holds
//    l(i, k) of its row, and warp w updates the tile columns j = k + 1 + w (mod 4) with l(j, k)
//    taken from lane j by a shuffle; a 128-thread barrier separates the pivots;
//  * the rows below, X <- X L_D^{-T}, one thread per row by forward substitution (the tile
//    is read by broadcast from shared memory);
//  * the trailing update of the rest of the leaf in 4 x 4 register blocks with 16-byte loads;
// the last two in the storage precision T.  S: column-major, ld L = a multiple of 4 above sz.
constexpr int LEAF_FUSED_MAX = 192;
constexpr int LP = 32;   // panel width of the leaf factorization
__host__ __device__ constexpr int leaf_ld(int sz) { return (sz + 4) / 4 * 4; }
constexpr int LEAF_DT = LP + 1;          // column stride of the FP64 tile

template <class T, class TT>
__device__ __forceinline__ void leaf_tile_chol4(T* S, int L, int t0, int nb, TT* D, T* dinv, int* status,
                                                int node) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;   // w < 4
    for (int k = 0; k < nb; ++k) {
        TT piv = D[k * LEAF_DT + k];
        if (!(piv > TT(0))) {        // indefinite or NaN pivot: record, keep values finite
            if (threadIdx.x == 0) atomicCAS(status, 0, node + 1);
            piv = TT(1);
        }
        const TT y = rsqrt_tile(piv);
        const TT lik = (lane > k && lane < nb) ? D[k * LEAF_DT + lane] * y : TT(0);
        for (int j = k + 1 + w; j < nb; j += 4) {
            const TT ljk = __shfl_sync(0xffffffffu, lik, j);
            if (lane >= j && lane < nb) D[j * LEAF_DT + lane] = fma(-lik, ljk, D[j * LEAF_DT + lane]);
        }
        if (w == 0) {
            if (lane == k) { S[t0 + k + (size_t)(t0 + k) * L] = (T)(piv * y); dinv[k] = (T)y; }
            else if (lane > k && lane < nb) S[t0 + lane + (size_t)(t0 + k) * L] = (T)lik;
        }
        asm volatile("bar.sync 1, 128;" ::: "memory");
    }
}

template <class T>
__global__ void __launch_bounds__(256) k_leaf_factor(const PotrfTask* __restrict__ tasks, int* status) {
    extern __shared__ __align__(16) unsigned char lf_smem[];
    __shared__ T dinv[LP];
    const PotrfTask tk = tasks[blockIdx.x];
    T* a = (T*)tk.a;
    const int sz = tk.nb, ld = tk.ld, L = leaf_ld(sz);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    T* S = (T*)lf_smem;
    using TT = typename TileType<T>::type;
    TT* D = (TT*)(lf_smem + ((size_t)sizeof(T) * sz * L + 15) / 16 * 16);   // 32 x 33 tile
    for (int j = warp; j < sz; j += 8)
        for (int i = j + lane; i < sz; i += 32) S[i + j * L] = a[i + (size_t)j * ld];
    __syncthreads();
    for (int t0 = 0; t0 < sz; t0 += LP) {
        const int nb = min(LP, sz - t0);
        for (int e = tid; e < LP * LP; e += blockDim.x) {
            const int i = e & 31, j = e >> 5;
            D[j * LEAF_DT + i] = (i < nb && j < nb && i >= j) ? (TT)S[t0 + i + (size_t)(t0 + j) * L] : TT(0);
        }
        __syncthreads();
        if (warp < 4) leaf_tile_chol4<T, TT>(S, L, t0, nb, D, dinv, status, tk.node);
        __syncthreads();
        const int r0 = t0 + nb, m = sz - r0;             // rows below the tile
        if (m <= 0) break;
        // X <- X L_D^{-T}: row i of X solves x L_D^T = b by forward substitution
        const T* Ld = S + t0 + (size_t)t0 * L;
        for (int i = tid; i < m; i += blockDim.x) {
            T* row = S + r0 + i + (size_t)t0 * L;
            T x[LP];
#pragma unroll
            for (int c = 0; c < LP; ++c) {
                if (c >= nb) break;
                T sacc = row[(size_t)c * L];
#pragma unroll
                for (int l = 0; l < c; ++l) sacc = fma(-x[l], Ld[c + (size_t)l * L], sacc);
                x[c] = sacc * dinv[c];
            }
#pragma unroll
            for (int c = 0; c < LP; ++c) {
                if (c >= nb) break;
                row[(size_t)c * L] = x[c];
            }
        }
        __syncthreads();
        // trailing update: S[i][j] -= sum_c X[i][c] X[j][c] for r0 <= j <= i < sz, 4 x 4 blocks
        // (r0 and L are multiples of 4: a block's four rows of a column are one 16-byte load;
        // rows past sz read the column's padding and are never written)
        const int mb = (m + 3) >> 2;                     // 4-row blocks
        const int nblk = mb * (mb + 1) / 2;              // lower-triangular block pairs (bi >= bj)
        for (int e = tid; e < nblk; e += blockDim.x) {
            int bi = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
            while ((bi + 1) * (bi + 2) / 2 <= e) ++bi;
            while (bi * (bi + 1) / 2 > e) --bi;
            const int bj = e - bi * (bi + 1) / 2;
            const int i0 = r0 + 4 * bi, j0 = r0 + 4 * bj;
            T acc[4][4];
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] = T(0);
            for (int c = 0; c < nb; ++c) {
                const T* col = S + (size_t)(t0 + c) * L;
                T xi[4], xj[4];
                if (sizeof(T) == 4) {
                    const float4 fi = *reinterpret_cast<const float4*>(col + i0);
                    const float4 fj = *reinterpret_cast<const float4*>(col + j0);
                    xi[0] = fi.x; xi[1] = fi.y; xi[2] = fi.z; xi[3] = fi.w;
                    xj[0] = fj.x; xj[1] = fj.y; xj[2] = fj.z; xj[3] = fj.w;
                } else {
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const double2 fi = *reinterpret_cast<const double2*>(col + i0 + 2 * h);
                        const double2 fj = *reinterpret_cast<const double2*>(col + j0 + 2 * h);
                        xi[2 * h] = fi.x; xi[2 * h + 1] = fi.y;
                        xj[2 * h] = fj.x; xj[2 * h + 1] = fj.y;
                    }
                }
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v) acc[u][v] = fma(xi[u], xj[v], acc[u][v]);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    const int i = i0 + u, j = j0 + v;
                    if (i < sz && j <= i) S[i + (size_t)j * L] -= acc[u][v];
                }
        }
        __syncthreads();
    }
    for (int j = warp; j < sz; j += 8)
        for (int i = j + lane; i < sz; i += 32) a[i + (size_t)j * ld] = S[i + j * L];
}

// X L^T = B for a block of rows (nrows <= 64) below a factored diagonal tile (in place).
// Thread (ty, tx) keeps rows ty + 16 p and columns tx + 16 q of X in registers; column j is
// scaled by the reciprocal pivot by its owners and published to shared memory, then every
// thread subtracts its contribution from the columns right of j (one barrier per column).
template <class T>
__global__ void __launch_bounds__(256) k_trsm_tile(const TrsmTask* __restrict__ tasks) {
    __shared__ T Ls[NB][NB + 1];
    __shared__ T dinv[NB];
    __shared__ T colj[2][TILE];
    const TrsmTask tk = tasks[blockIdx.x];
    const T* L = (const T*)tk.L;
    T* B = (T*)tk.B;
    const int nb = tk.nb, nr = tk.nrows;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
        const int i = e & (NB - 1), j = e >> 6;
        Ls[i][j] = (i < nb && j < nb && i >= j) ? L[i + (size_t)j * tk.ldl] : T(0);
    }
    __syncthreads();
    if (threadIdx.x < nb) dinv[threadIdx.x] = T(1) / Ls[threadIdx.x][threadIdx.x];
    T x[4][4];
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int i = ty + 16 * p, j = tx + 16 * q;
            x[p][q] = (i < nr && j < nb) ? B[i + (size_t)j * tk.ldb] : T(0);
        }
    __syncthreads();
    for (int j = 0; j < nb; ++j) {
        const int buf = j & 1, jq = j >> 4;
        if (tx == (j & 15)) {
            const T di = dinv[j];
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (q == jq) {
                        x[p][q] *= di;
                        colj[buf][ty + 16 * p] = x[p][q];
                    }
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (16 * q + 15 <= j) continue;           // whole warp left of column j + 1
            const int l = tx + 16 * q;
            const T lj = (l > j && l < nb) ? Ls[l][j] : T(0);
#pragma unroll
            for (int p = 0; p < 4; ++p) x[p][q] = fma(-colj[buf][ty + 16 * p], lj, x[p][q]);
        }
    }
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int i = ty + 16 * p, j = tx + 16 * q;
            if (i < nr && j < nb) B[i + (size_t)j * tk.ldb] = x[p][q];
        }
}

// ------------------------------------------------------------------ 64x64 tile product core
// acc[a][b] = sum_l A[ty + 16a, l] * B[tx + 16b, l] over l < K, rows masked by m / n.
template <class T>
__device__ __forceinline__ void tile_nt(const T* __restrict__ A, int lda, int m, const T* __restrict__ B, int ldb,
                                        int n, int K, T (&acc)[4][4], T (*As)[TILE + 1], T (*Bs)[TILE + 1]) {
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
    for (int k0 = 0; k0 < K; k0 += KCH) {
        for (int e = tid; e < KCH * TILE; e += 256) {
            int r = e % TILE, kk = e / TILE;
            int l = k0 + kk;
            As[kk][r] = (r < m && l < K) ? A[r + (size_t)l * lda] : T(0);
            Bs[kk][r] = (r < n && l < K) ? B[r + (size_t)l * ldb] : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < KCH; ++kk) {
            T av[4], bv[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) av[a] = As[kk][ty + 16 * a];
#pragma unroll
            for (int b = 0; b < 4; ++b) bv[b] = Bs[kk][tx + 16 * b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
        }
        __syncthreads();
    }
}

template <class T>
__global__ void __launch_bounds__(256) k_gemm_tile(const GemmTask* __restrict__ tasks) {
    __shared__ T As[KCH][TILE + 1];
    __shared__ T Bs[KCH][TILE + 1];
    const GemmTask tk = tasks[blockIdx.x];
    T acc[4][4];
    tile_nt<T>((const T*)tk.A, tk.lda, tk.m, (const T*)tk.B, tk.ldb, tk.n, tk.K, acc, As, Bs);
    T* C = (T*)tk.C;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            int i = ty + 16 * a, j = tx + 16 * b;
            if (i < tk.m && j < tk.n && (!tk.lower || i + tk.moff >= j)) C[i + (size_t)j * tk.ldc] -= acc[a][b];
        }
}

// ------------------------------------------------------------------ extend-add (push form)
// For descendant k: S = L^O_k(pr0:pr1,:) L^O_k(pc0:pc1,:)^T, lower part (row position >=
// column position), subtracted from ancestor j's storage at (row R_k[q], column R_k[p]).
template <class T>
__global__ void __launch_bounds__(256) k_push(const PushTask* __restrict__ tasks, const LoOp* __restrict__ lo,
                                              const NodeTgt* __restrict__ tgts, const int32_t* __restrict__ rows,
                                              const long long* __restrict__ rows_ptr,
                                              const LeafMap* __restrict__ leafmap, T* __restrict__ arena) {
    __shared__ T As[KCH][TILE + 1];
    __shared__ T Bs[KCH][TILE + 1];
    __shared__ long long rpart[TILE], cpart[TILE];
    __shared__ long long rleaf[TILE], cleaf[TILE];
    const PushTask tk = tasks[blockIdx.x];
    const LoOp op = lo[tk.k];
    const NodeTgt tg = tgts[tk.j];
    if (tg.kind == 3 || op.K == 0) return;
    const int32_t* Rk = rows + rows_ptr[tk.k];
    const int m = tk.pr1 - tk.pr0, n = tk.pc1 - tk.pc0;
    for (int i = threadIdx.x; i < TILE; i += blockDim.x) {
        long long rp = -1, rl = -1;
        if (i < m) {
            long long g = Rk[tk.pr0 + i];
            bool inC = g < tg.c0 + tg.c;
            if (tg.kind == 0) {
                rp = inC ? g - tg.c0 : tg.c + lower_bound_i32(rows + tg.rows_off, tg.r, (int32_t)g);
            } else if (inC) {
                if (tg.kind == 1) rp = g - tg.c0;
                else { LeafMap lm = leafmap[g]; rp = g - lm.lo; rl = lm.lo; }
            }
        }
        rpart[i] = rp;
        rleaf[i] = rl;
        long long cp = -1, cl = -1;
        if (i < n) {
            long long g = Rk[tk.pc0 + i];
            if (tg.kind == 0 || tg.kind == 1) cp = (g - tg.c0) * (long long)tg.ld;
            else { LeafMap lm = leafmap[g]; cp = lm.off + (g - lm.lo) * (long long)lm.size; cl = lm.lo; }
        }
        cpart[i] = cp;
        cleaf[i] = cl;
    }
    __syncthreads();
    const T* base = (const T*)op.base;
    T acc[4][4];
    tile_nt<T>(base + tk.pr0, op.ld, m, base + tk.pc0, op.ld, n, op.K, acc, As, Bs);
    T* dst = tg.kind == 2 ? arena : (T*)tg.base;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            int i = ty + 16 * a, j = tx + 16 * b;
            if (i >= m || j >= n) continue;
            if (tk.pr0 + i < tk.pc0 + j) continue;                 // upper part
            long long rp = rpart[i];
            if (rp < 0) continue;
            if (tg.kind == 2 && rleaf[i] != cleaf[j]) continue;    // not inside one leaf block
            atomic_add(dst + rp + cpart[j], -acc[a][b]);
        }
}

// ------------------------------------------------------------------ thin products
// TN products Z = A^T Y: k_tn1 (one right-hand side, the preconditioner apply) below, k_tn_s
// (up to 64 columns, staged through shared memory) further down; NN products Y += A Z: k_nn.
constexpr int TN_COLS = 32;
// 16 consecutive elements from a 16-byte aligned address, as 16-byte vector loads
__device__ __forceinline__ void load_row16(const float* y, float (&v)[16]) {
    const float4* p = reinterpret_cast<const float4*>(y);
#pragma unroll
    for (int h = 0; h < 4; ++h) {
        const float4 f = p[h];
        v[4 * h] = f.x; v[4 * h + 1] = f.y; v[4 * h + 2] = f.z; v[4 * h + 3] = f.w;
    }
}
__device__ __forceinline__ void load_row16(const double* y, double (&v)[16]) {
    const double2* p = reinterpret_cast<const double2*>(y);
#pragma unroll
    for (int h = 0; h < 8; ++h) {
        const double2 f = p[h];
        v[2 * h] = f.x; v[2 * h + 1] = f.y;
    }
}
// TN product for one right-hand side (N = 1, the preconditioner apply): one CTA per (task, 32-
// column tile, row split).  The gathered y values of a 512-row chunk are staged in shared memory
// once for the CTA; warp w then takes columns 4w .. 4w + 3 together (four independent
// accumulators, lanes down the rows: coalesced reads of A) and reduces them with shuffles.
// With tk.nsplit > 1, CTA z sums rows [z rps, (z + 1) rps) into part[z][32] and the last CTA to
// arrive adds the partial sums in ascending z (deterministic) and resets its counter.
constexpr int TN1_CHUNK = 512;
template <class T>
__global__ void __launch_bounds__(256) k_tn1(const TnTask* __restrict__ tasks) {
    __shared__ T ys[TN1_CHUNK];
    __shared__ int last;
    const TnTask tk = tasks[blockIdx.x];
    if ((int)blockIdx.z >= tk.nsplit) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int rb = (int)blockIdx.z * tk.rps;
    const int re = tk.nsplit > 1 ? min(tk.nrow, rb + tk.rps) : tk.nrow;
    const T* Y = (const T*)tk.Y;
    T* part = (T*)tk.part;
    const int tt0 = 4 * warp;                          // this warp's first column of the tile
    const T* A = (const T*)tk.A + (size_t)(tk.t0 + tt0) * tk.lda;
    bool ok[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) ok[u] = tk.t0 + tt0 + u < tk.K;
    T acc[4] = {T(0), T(0), T(0), T(0)};
    for (int c0 = rb; c0 < re; c0 += TN1_CHUNK) {
        const int cn = min(TN1_CHUNK, re - c0);
        __syncthreads();
        for (int i = threadIdx.x; i < cn; i += blockDim.x) {
            const int yr = (tk.ymap ? tk.ymap[c0 + i] : c0 + i) + tk.yoff;
            ys[i] = Y[(size_t)yr * tk.ldy];
        }
        __syncthreads();
        if (ok[0]) {
#pragma unroll 2
            for (int i = lane; i < cn; i += 32) {
                const int ar = (tk.amap ? tk.amap[c0 + i] : c0 + i) + tk.aoff;
                const T yv = ys[i];
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (ok[u]) acc[u] = fma(A[(size_t)u * tk.lda + ar], yv, acc[u]);
            }
        }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc[u] += __shfl_xor_sync(0xffffffffu, acc[u], o);
    if (lane == 0) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (!ok[u]) continue;
            const int tt = tt0 + u;
            if (tk.nsplit == 1) {
                T* z = (T*)tk.Z + (size_t)(tk.t0 + tt) * tk.ldz;
                *z = tk.beta != 0.0 ? (T)tk.beta * *z + (T)tk.alpha * acc[u] : (T)tk.alpha * acc[u];
            } else {
                part[(size_t)blockIdx.z * TN_COLS + tt] = acc[u];
            }
        }
    }
    if (tk.nsplit == 1) return;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(tk.cnt, 1u) == (unsigned)(tk.nsplit - 1);
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (threadIdx.x < TN_COLS && tk.t0 + (int)threadIdx.x < tk.K) {
        T a = T(0);
        for (int zz = 0; zz < tk.nsplit; ++zz) a += __ldcg(part + (size_t)zz * TN_COLS + threadIdx.x);
        T* z = (T*)tk.Z + (size_t)(tk.t0 + threadIdx.x) * tk.ldz;
        *z = tk.beta != 0.0 ? (T)tk.beta * *z + (T)tk.alpha * a : (T)tk.alpha * a;
    }
    if (threadIdx.x == 0) *tk.cnt = 0u;
}

// ------------------------------------------------------------------ staged TN product (factorization)
// Z[t, :] = beta Z[t, :] + alpha sum_i A[arow_i, t] Y[yrow_i, :] for one 64-column tile of A
// (t0 .. t0 + 63) and up to 64 columns of Y in one CTA, so every element of A is read from
// memory once.  Rows stream through shared memory in chunks of 32 with cp.async double
// buffering: the A chunk is read down its columns (a warp reads 32 consecutive rows of one
// column, 128 contiguous bytes for FP32) into As[t][r], the Y chunk row by row (the gathered
// rows are contiguous N-vectors, copied 16 bytes at a time when aligned) into Ys[r][c].
// Thread (tg, cg) owns TT columns of A and 4 columns of Y (NP = N padded to 16, 32 or 64;
// TT = NP / 16) and accumulates over the chunk's rows from shared memory, RV rows per step
// (one 16-byte load of As per column and of Ys per row: 64 multiply-adds per 8 loads in
// FP32), so no cross-thread reduction is needed; rows past the chunk's end are zero-filled.
// With tk.nsplit > 1 CTA z takes rows [z rps, (z + 1) rps) and writes its partial sums to
// part[z][64][N]; the last CTA to arrive (counter cnt[y]) adds them in ascending z
// (deterministic), writes Z and resets the counter.
constexpr int TS_COLS = 64;
constexpr int TS_ROWS = 32;
template <class T>
__host__ __device__ constexpr size_t ts_smem_bytes(int np) {
    return sizeof(T) * ((size_t)2 * TS_COLS * (TS_ROWS + 4) + (size_t)2 * TS_ROWS * (np + 4));
}
__device__ __forceinline__ void cp_async4(void* sdst, const void* gsrc) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" :: "r"((uint32_t)__cvta_generic_to_shared(sdst)), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async8(void* sdst, const void* gsrc) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" :: "r"((uint32_t)__cvta_generic_to_shared(sdst)), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" :: "r"((uint32_t)__cvta_generic_to_shared(sdst)), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" :: "n"(N) : "memory"); }

template <class T, int NP>
__global__ void __launch_bounds__(256) k_tn_s(const TnTask* __restrict__ tasks) {
    extern __shared__ __align__(16) unsigned char ts_smem[];
    constexpr int AST = TS_ROWS + 4;       // As[t][r]: a column of the chunk per row of As (16-byte rows)
    constexpr int YST = NP + 4;            // Ys[r][c]: 16-byte aligned rows
    constexpr int CG = NP / 4;             // column groups of 4
    constexpr int TT = TS_COLS * CG / 256; // columns of A per thread
    constexpr int RV = 16 / (int)sizeof(T);   // rows per step (one 16-byte load)
    T* As = (T*)ts_smem;
    T* Ys = As + 2 * TS_COLS * AST;
    __shared__ int last;
    const TnTask tk = tasks[blockIdx.x];
    const int cb = blockIdx.y * 64;                     // 64-column chunk of Y and Z
    const int nc = min(64, tk.N - cb);
    if (nc <= 0 || (int)blockIdx.z >= tk.nsplit) return;
    const int tid = threadIdx.x;
    const int rb = (int)blockIdx.z * tk.rps;
    const int re = tk.nsplit > 1 ? min(tk.nrow, rb + tk.rps) : tk.nrow;
    const int kc = min(TS_COLS, tk.K - tk.t0);          // valid columns of this tile
    const T* A = (const T*)tk.A + (size_t)tk.t0 * tk.lda;
    const T* Y = (const T*)tk.Y + cb;
    constexpr int VW = 16 / (int)sizeof(T);             // elements per 16-byte copy
    const bool yvec = (nc % VW) == 0 && (tk.ldy % VW) == 0 && (((uintptr_t)Y) & 15) == 0;
    auto issue = [&](int r0, int buf) {
        const int rc = min(TS_ROWS, re - r0);
        const int rc4 = (rc + RV - 1) / RV * RV;
        T* as = As + buf * TS_COLS * AST;
        T* ys = Ys + buf * TS_ROWS * YST;
        for (int e = tid; e < TS_COLS * TS_ROWS; e += 256) {
            const int t = e / TS_ROWS, r = e % TS_ROWS;
            if (t < kc && r < rc) {
                const int i = r0 + r;
                const int ar = (tk.amap ? tk.amap[i] : i) + tk.aoff;
                const T* src = A + (size_t)t * tk.lda + ar;
                if (sizeof(T) == 8) cp_async8(as + t * AST + r, src);
                else cp_async4(as + t * AST + r, src);
            } else if (r >= rc && r < rc4) {
                as[t * AST + r] = T(0);
            }
        }
        if (rc4 > rc)
            for (int e = tid; e < (rc4 - rc) * NP; e += 256) ys[(rc + e / NP) * YST + e % NP] = T(0);
        if (yvec) {
            const int per = nc / VW;
            for (int e = tid; e < TS_ROWS * per; e += 256) {
                const int r = e / per, q = e % per;
                if (r < rc) {
                    const int i = r0 + r;
                    const int yr = (tk.ymap ? tk.ymap[i] : i) + tk.yoff;
                    cp_async16(ys + r * YST + q * VW, Y + (size_t)yr * tk.ldy + q * VW);
                }
            }
        } else {
            for (int e = tid; e < TS_ROWS * nc; e += 256) {
                const int r = e / nc, c = e % nc;
                if (r < rc) {
                    const int i = r0 + r;
                    const int yr = (tk.ymap ? tk.ymap[i] : i) + tk.yoff;
                    if (sizeof(T) == 8) cp_async8(ys + r * YST + c, Y + (size_t)yr * tk.ldy + c);
                    else cp_async4(ys + r * YST + c, Y + (size_t)yr * tk.ldy + c);
                }
            }
        }
        cp_async_commit();
    };
    const int cg = tid % CG, tg = tid / CG;
    T acc[TT][4];
#pragma unroll
    for (int u = 0; u < TT; ++u)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[u][q] = T(0);
    const int nch = (re - rb + TS_ROWS - 1) / TS_ROWS;
    if (nch > 0) issue(rb, 0);
    for (int ci = 0; ci < nch; ++ci) {
        const int buf = ci & 1;
        if (ci + 1 < nch) { issue(rb + (ci + 1) * TS_ROWS, buf ^ 1); cp_async_wait<1>(); }
        else cp_async_wait<0>();
        __syncthreads();
        const int rc = min(TS_ROWS, re - rb - ci * TS_ROWS);
        const T* as = As + buf * TS_COLS * AST + (tg * TT) * AST;
        const T* ys = Ys + buf * TS_ROWS * YST + cg * 4;
        for (int r = 0; r < rc; r += RV) {
            T yv[RV][4], av[TT][RV];
#pragma unroll
            for (int h = 0; h < RV; ++h) {
                if (sizeof(T) == 4) {
                    const float4 f = *reinterpret_cast<const float4*>(ys + (r + h) * YST);
                    yv[h][0] = f.x; yv[h][1] = f.y; yv[h][2] = f.z; yv[h][3] = f.w;
                } else {
                    const double2 f0 = *reinterpret_cast<const double2*>(ys + (r + h) * YST);
                    const double2 f1 = *reinterpret_cast<const double2*>(ys + (r + h) * YST + 2);
                    yv[h][0] = f0.x; yv[h][1] = f0.y; yv[h][2] = f1.x; yv[h][3] = f1.y;
                }
            }
#pragma unroll
            for (int u = 0; u < TT; ++u) {
                if (sizeof(T) == 4) {
                    const float4 f = *reinterpret_cast<const float4*>(as + u * AST + r);
                    av[u][0] = f.x; av[u][1] = f.y; av[u][2] = f.z; av[u][3] = f.w;
                } else {
                    const double2 f = *reinterpret_cast<const double2*>(as + u * AST + r);
                    av[u][0] = f.x; av[u][1] = f.y;
                }
            }
#pragma unroll
            for (int h = 0; h < RV; ++h)
#pragma unroll
                for (int u = 0; u < TT; ++u)
#pragma unroll
                    for (int q = 0; q < 4; ++q) acc[u][q] = fma(av[u][h], yv[h][q], acc[u][q]);
        }
        __syncthreads();
    }
    const int c0 = cg * 4;
    if (tk.nsplit == 1) {
#pragma unroll
        for (int u = 0; u < TT; ++u) {
            const int t = tg * TT + u;
            if (t >= kc) continue;
            T* z = (T*)tk.Z + (size_t)(tk.t0 + t) * tk.ldz + cb;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int c = c0 + q;
                if (c >= nc) break;
                z[c] = tk.beta != 0.0 ? (T)tk.beta * z[c] + (T)tk.alpha * acc[u][q] : (T)tk.alpha * acc[u][q];
            }
        }
        return;
    }
    // partial sums of this row range: part[z][t][cb + c], row length N
    T* part = (T*)tk.part;
#pragma unroll
    for (int u = 0; u < TT; ++u) {
        const int t = tg * TT + u;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int c = c0 + q;
            if (c < nc) part[((size_t)blockIdx.z * TS_COLS + t) * tk.N + cb + c] = acc[u][q];
        }
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) last = atomicAdd(tk.cnt + blockIdx.y, 1u) == (unsigned)(tk.nsplit - 1);
    __syncthreads();
    if (!last) return;
    __threadfence();
    for (int e = tid; e < kc * nc; e += 256) {
        const int t = e / nc, c = e % nc;
        T s = T(0);
        for (int zz = 0; zz < tk.nsplit; ++zz) s += __ldcg(part + ((size_t)zz * TS_COLS + t) * tk.N + cb + c);
        T* z = (T*)tk.Z + (size_t)(tk.t0 + t) * tk.ldz + cb + c;
        *z = tk.beta != 0.0 ? (T)tk.beta * *z + (T)tk.alpha * s : (T)tk.alpha * s;
    }
    if (tid == 0) tk.cnt[blockIdx.y] = 0u;
}

// One CTA of 128 threads per (task, 128-row chunk, 16-column chunk); a thread owns one
// row and its 16 outputs, so each element of A is loaded once.
constexpr int NN_ROWS = 128;
template <class T>
__global__ void __launch_bounds__(NN_ROWS) k_nn(const NnTask* __restrict__ tasks) {
    __shared__ __align__(16) T Zs[64][16];   // read by every thread (broadcast) as 16-byte vectors
    const NnTask tk = tasks[blockIdx.x];
    const int c0 = blockIdx.y * 16;
    const int nc = min(16, tk.N - c0);
    if (nc <= 0) return;
    const int i = tk.row0 + threadIdx.x;
    const bool active = i < tk.nrow;
    const T* A = (const T*)tk.A;
    const T* Z = (const T*)tk.Z;
    int ar = 0;
    if (active) ar = (tk.amap ? tk.amap[i] : i) + tk.aoff;
    T acc[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) acc[q] = T(0);
    for (int l0 = 0; l0 < tk.K; l0 += 64) {
        const int lk = min(64, tk.K - l0);
        __syncthreads();
        for (int e = threadIdx.x; e < 64 * 16; e += blockDim.x) {
            const int l = e >> 4, c = e & 15;
            Zs[l][c] = (l < lk && c < nc) ? Z[(size_t)(l0 + l) * tk.ldz + c0 + c] : T(0);
        }
        __syncthreads();
        if (active) {
            if (nc == 1) {
                for (int l = 0; l < lk; ++l) acc[0] = fma(A[ar + (size_t)(l0 + l) * tk.lda], Zs[l][0], acc[0]);
            } else {
#pragma unroll 4
                for (int l = 0; l < lk; ++l) {
                    const T a = A[ar + (size_t)(l0 + l) * tk.lda];
                    T zv[16];
                    load_row16(&Zs[l][0], zv);
#pragma unroll
                    for (int q = 0; q < 16; ++q) acc[q] = fma(a, zv[q], acc[q]);
                }
            }
        }
    }
    if (!active) return;
    const int yr = (tk.ymap ? tk.ymap[i] : i) + tk.yoff;
    T* y = (T*)tk.Y + (size_t)yr * tk.ldy + c0;
    const T alpha = (T)tk.alpha;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        if (q >= nc) break;
        if (tk.atomic) atomic_add(y + q, alpha * acc[q]);
        else y[q] += alpha * acc[q];
    }
}

// Y[i, :] = alpha * sum_e v[e] X[ci[e], :] for 16 rows x 16 columns per CTA.
template <class T>
__global__ void k_csr_mm(const CsrTask* __restrict__ tasks) {
    const CsrTask tk = tasks[blockIdx.x];
    const int c0 = blockIdx.y * 16;
    const int nc = min(16, tk.N - c0);
    if (nc <= 0) return;
    const int i = tk.row0 + (threadIdx.x >> 4), c = threadIdx.x & 15;
    if (i >= tk.blk.nrows || c >= nc) return;
    const T* X = (const T*)tk.X;
    T s = T(0);
    for (int q = tk.blk.rp[i]; q < tk.blk.rp[i + 1]; ++q)
        s = fma((T)tk.blk.v[q], X[(size_t)tk.blk.ci[q] * tk.ldx + c0 + c], s);
    const long long orow = tk.rmap ? tk.rmap[i] : i;
    const long long ocol = tk.cmap ? tk.cmap[c0 + c] : c0 + c;
    if (tk.lower && ocol < orow) return;
    T* y = (T*)tk.Y + orow * tk.ldy + ocol;
    const T v = (T)tk.alpha * s;
    if (tk.mode == 0) *y = v;
    else if (tk.mode == 1) *y += v;
    else atomicAdd(y, v);
}

// ------------------------------------------------------------------ dense triangular solves with many RHS
// X (c x N, row-major) <- L^{-1} X or L^{-T} X, one CTA per (task, CW-column chunk), c <= SOLVE_MAX.
// Blocked by 32 rows: a warp solves each column of the 32 x 32 diagonal tile with
// shuffles, then the CTA updates the remaining rows with the solved block.
template <class T, int CW>
__global__ void __launch_bounds__(256) k_trsv_subst(const TrsvTask* __restrict__ tasks) {
    __shared__ T Xs[SOLVE_MAX][CW + 1];
    __shared__ T Lt[32][33];
    __shared__ T dinv[32];
    const TrsvTask tk = tasks[blockIdx.x];
    const T* L = (const T*)tk.L;
    T* X = (T*)tk.X;
    const int c = tk.c, ld = tk.ld, transpose = tk.transpose == 1;
    const int c0 = blockIdx.y * CW;
    const int nc = min(CW, tk.N - c0);
    if (nc <= 0) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int e = tid; e < c * CW; e += blockDim.x) {
        int i = e / CW, q = e % CW;
        if (tk.transpose == 2) Xs[i][q] = (q < nc && i == c0 + q) ? T(1) : T(0);   // invert: X = L^{-1} I
        else Xs[i][q] = q < nc ? X[(size_t)i * tk.ldx + c0 + q] : T(0);
    }
    const int nb = (c + 31) >> 5;
    constexpr int G = CW >= 4 ? 4 : CW;          // columns per thread in the update
    constexpr int NG = CW / G;                    // column groups
    for (int bi = 0; bi < nb; ++bi) {
        const int b = transpose ? nb - 1 - bi : bi;
        const int r0 = b * 32, w = min(32, c - r0);
        __syncthreads();
        for (int e = tid; e < 32 * 32; e += blockDim.x) {
            int i = e & 31, j = e >> 5;
            Lt[i][j] = (i < w && j < w && i >= j) ? L[(r0 + i) + (size_t)(r0 + j) * ld] : T(0);
        }
        __syncthreads();
        if (tid < w) dinv[tid] = T(1) / Lt[tid][tid];
        __syncthreads();
        for (int q = warp; q < nc; q += 8) {
            T x = lane < w ? Xs[r0 + lane][q] : T(0);
            if (!transpose) {
                for (int k2 = 0; k2 < w; ++k2) {
                    if (lane == k2) x *= dinv[k2];
                    const T xk = __shfl_sync(0xffffffffu, x, k2);
                    if (lane > k2) x -= Lt[lane][k2] * xk;
                }
            } else {
                for (int k2 = w - 1; k2 >= 0; --k2) {
                    if (lane == k2) x *= dinv[k2];
                    const T xk = __shfl_sync(0xffffffffu, x, k2);
                    if (lane < k2) x -= Lt[k2][lane] * xk;
                }
            }
            if (lane < w) Xs[r0 + lane][q] = x;
        }
        __syncthreads();
        const int lo = transpose ? 0 : r0 + w;
        const int cnt = transpose ? r0 : c - r0 - w;
        for (int e = tid; e < cnt * NG; e += blockDim.x) {
            const int i = lo + e / NG, g0 = (e % NG) * G;
            if (g0 >= nc) continue;
            T a[G];
#pragma unroll
            for (int u = 0; u < G; ++u) a[u] = T(0);
#pragma unroll 8
            for (int k2 = 0; k2 < w; ++k2) {
                const T l = transpose ? L[(r0 + k2) + (size_t)i * ld] : L[i + (size_t)(r0 + k2) * ld];
#pragma unroll
                for (int u = 0; u < G; ++u) a[u] = fma(l, Xs[r0 + k2][g0 + u], a[u]);
            }
#pragma unroll
            for (int u = 0; u < G; ++u) Xs[i][g0 + u] -= a[u];
        }
    }
    __syncthreads();
    for (int e = tid; e < c * CW; e += blockDim.x) {
        int i = e / CW, q = e % CW;
        if (q < nc) X[(size_t)i * tk.ldx + c0 + q] = Xs[i][q];
    }
}

// ------------------------------------------------------------------ triangular solves by explicit inverse
// Xb (c x CW rows in shared memory) <- Linv Xb or Linv^T Xb, Linv the row-major inverse
// of a lower-triangular diagonal block (c <= SOLVE_MAX); the result goes through Zs.
// Forward: a warp per output row, lanes along the row (coalesced); transposed: a
// thread per output, reading one row of Linv per step (coalesced).  Ends synced.
template <class T, int CW>
__device__ __forceinline__ void trmv_inv(const T* __restrict__ Li, int c, T* Xb, T* Zs, bool transpose) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (!transpose) {
        // a warp takes four rows at a time (their loads are independent)
        const int nw = blockDim.x >> 5;
        for (int i0 = 4 * warp; i0 < c; i0 += 4 * nw) {
            T acc[4][CW];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int q = 0; q < CW; ++q) acc[r][q] = T(0);
            const int iend = min(c - 1, i0 + 3);
            for (int kk = lane; kk <= iend; kk += 32) {
                T v[4];
#pragma unroll
                for (int r = 0; r < 4; ++r) v[r] = (i0 + r <= iend && kk <= i0 + r) ? Li[(size_t)(i0 + r) * c + kk] : T(0);
#pragma unroll
                for (int q = 0; q < CW; ++q) {
                    const T xq = Xb[(size_t)kk * CW + q];
#pragma unroll
                    for (int r = 0; r < 4; ++r) acc[r][q] = fma(v[r], xq, acc[r][q]);
                }
            }
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int q = 0; q < CW; ++q) {
                    T v = acc[r][q];
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                    if (lane == 0 && i0 + r <= iend) Zs[(size_t)(i0 + r) * CW + q] = v;
                }
        }
    } else {
        for (int i = tid; i < c; i += blockDim.x) {
            T acc[CW];
#pragma unroll
            for (int q = 0; q < CW; ++q) acc[q] = T(0);
#pragma unroll 8
            for (int kk = i; kk < c; ++kk) {
                const T v = Li[(size_t)kk * c + i];
#pragma unroll
                for (int q = 0; q < CW; ++q) acc[q] = fma(v, Xb[(size_t)kk * CW + q], acc[q]);
            }
#pragma unroll
            for (int q = 0; q < CW; ++q) Zs[(size_t)i * CW + q] = acc[q];
        }
    }
    __syncthreads();
    for (int e = tid; e < c * CW; e += blockDim.x) Xb[e] = Zs[e];
    __syncthreads();
}

// X (c x N, row-major) <- Linv X or Linv^T X for a batch of small diagonal blocks
// (TrsvTask.L = row-major inverse), one CTA per (task, CW-column chunk).
template <class T, int CW>
__global__ void __launch_bounds__(256) k_trsv(const TrsvTask* __restrict__ tasks) {
    __shared__ T Xs[SOLVE_MAX * CW];
    __shared__ T Zs[SOLVE_MAX * CW];
    const TrsvTask tk = tasks[blockIdx.x];
    const int c0 = blockIdx.y * CW;
    const int nc = min(CW, tk.N - c0);
    if (nc <= 0) return;
    T* X = (T*)tk.X;
    for (int e = threadIdx.x; e < tk.c * CW; e += blockDim.x) {
        const int i = e / CW, q = e % CW;
        Xs[e] = q < nc ? X[(size_t)i * tk.ldx + c0 + q] : T(0);
    }
    __syncthreads();
    trmv_inv<T, CW>((const T*)tk.L, tk.c, Xs, Zs, tk.transpose == 1);
    for (int e = threadIdx.x; e < tk.c * CW; e += blockDim.x) {
        const int i = e / CW, q = e % CW;
        if (q < nc) X[(size_t)i * tk.ldx + c0 + q] = Xs[e];
    }
}

// X (c x N, row-major) <- Linv X or Linv^T X, Linv the row-major inverse of a lower triangular
// block (c <= SOLVE_MAX, entries above its diagonal ignored): one CTA per (task, 64 columns).
// The CTA keeps its c x 64 slice of X in shared memory and runs 64 x 64 output tiles as a small
// GEMM over the 64 x 64 tiles of Linv on the triangle's side, each thread a 4 x 4 register block;
// Linv tiles are staged transposed (column kk of the tile contiguous) so both operands are read
// as 16-byte vectors.  Output tiles go in the order that leaves their inputs untouched (last
// tile first for Linv, first tile first for Linv^T), so X is updated in place.
constexpr int TT_COLS = 64, TT_TILE = 64, TT_LPAD = TT_TILE + 4;
template <class T>
constexpr size_t tt_smem_bytes() { return sizeof(T) * ((size_t)SOLVE_MAX * TT_COLS + (size_t)TT_TILE * TT_LPAD); }
template <class T>
__global__ void __launch_bounds__(256) k_trsv_tile(const TrsvTask* __restrict__ tasks) {
    extern __shared__ __align__(16) unsigned char tt_smem[];
    T* Xs = (T*)tt_smem;                               // c x 64
    T* Ls = Xs + (size_t)SOLVE_MAX * TT_COLS;          // [kk][ii], 64 x TT_LPAD
    const TrsvTask tk = tasks[blockIdx.x];
    const int c0 = blockIdx.y * TT_COLS;
    const int nc = min(TT_COLS, tk.N - c0);
    if (nc <= 0) return;
    const int c = tk.c;
    const bool tr = tk.transpose == 1;
    const T* Li = (const T*)tk.L;
    T* X = (T*)tk.X;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    for (int e = tid; e < c * TT_COLS; e += blockDim.x) {
        const int i = e >> 6, q = e & 63;
        Xs[e] = q < nc ? X[(size_t)i * tk.ldx + c0 + q] : T(0);
    }
    const int nt = (c + TT_TILE - 1) / TT_TILE;
    for (int it = 0; it < nt; ++it) {
        const int I = tr ? it : nt - 1 - it;
        const int i0 = I * TT_TILE;
        T acc[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
        const int kb = tr ? I : 0, ke = tr ? nt - 1 : I;
        for (int K = kb; K <= ke; ++K) {
            const int k0 = K * TT_TILE;
            __syncthreads();   // Ls free (and Xs written) before the next tile
            for (int e = tid; e < TT_TILE * TT_TILE; e += blockDim.x) {
                // element (ii, kk) of the operator tile: Linv(i, k) or Linv(k, i), 0 above the diagonal
                int ii, kk;
                T v = T(0);
                if (!tr) {
                    ii = e >> 6; kk = e & 63;    // reads along a row of Linv
                    const int i = i0 + ii, k = k0 + kk;
                    if (i < c && k <= i) v = Li[(size_t)i * c + k];
                } else {
                    kk = e >> 6; ii = e & 63;    // reads along a row of Linv (row k)
                    const int i = i0 + ii, k = k0 + kk;
                    if (k < c && i <= k) v = Li[(size_t)k * c + i];
                }
                Ls[kk * TT_LPAD + ii] = v;
            }
            __syncthreads();
            const int kn = min(TT_TILE, c - k0);
            for (int kk = 0; kk < kn; ++kk) {
                T a[4], x[4];
#pragma unroll
                for (int r = 0; r < 4; ++r) a[r] = Ls[kk * TT_LPAD + ty * 4 + r];
#pragma unroll
                for (int q = 0; q < 4; ++q) x[q] = Xs[(size_t)(k0 + kk) * TT_COLS + tx * 4 + q];
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int q = 0; q < 4; ++q) acc[r][q] = fma(a[r], x[q], acc[r][q]);
            }
        }
        __syncthreads();   // every read of this tile's rows of X is done
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int i = i0 + ty * 4 + r;
            if (i < c)
#pragma unroll
                for (int q = 0; q < 4; ++q) Xs[(size_t)i * TT_COLS + tx * 4 + q] = acc[r][q];
        }
    }
    __syncthreads();
    for (int e = tid; e < c * TT_COLS; e += blockDim.x) {
        const int i = e >> 6, q = e & 63;
        if (q < nc) X[(size_t)i * tk.ldx + c0 + q] = Xs[e];
    }
}

// ------------------------------------------------------------------ persistent hierarchical solve
// One CTA per (task, CW-column chunk) walks a diagonal block's whole action list
// (Alg. 4 in order) with the right-hand side block (c x CW) staged in dynamic
// shared memory; the low-rank products go through a shared Z of 512 x CW.
constexpr int HS_ZROWS = 512;
constexpr int HS_THREADS = 512;
template <class T, int CW>
__global__ void __launch_bounds__(HS_THREADS) k_hsolve(const HTask* __restrict__ tasks) {
    extern __shared__ __align__(16) unsigned char hs_smem[];
    const HTask tk = tasks[blockIdx.x];
    const int c0 = blockIdx.y * CW;
    const int nc = min(CW, tk.N - c0);
    if (nc <= 0) return;
    T* Xs = (T*)hs_smem;                       // c x CW
    T* Zs = Xs + (size_t)tk.c * CW;            // HS_ZROWS x CW
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    T* X = (T*)tk.X;
    for (int e = tid; e < tk.c * CW; e += blockDim.x) {
        const int i = e / CW, q = e % CW;
        Xs[e] = q < nc ? X[(size_t)i * tk.ldx + c0 + q] : T(0);
    }
    __syncthreads();
    HAct nxt = tk.nact > 0 ? tk.acts[0] : HAct{};
    for (long long ai = 0; ai < tk.nact; ++ai) {
        const HAct a = nxt;                       // the next record is fetched while this one runs
        if (ai + 1 < tk.nact) nxt = tk.acts[ai + 1];
        if (a.type == HA_TRSV) {
            trmv_inv<T, CW>((const T*)a.A1, a.no, Xs + (size_t)a.o0 * CW, Zs, tk.transpose != 0);
        } else if (a.type == HA_LR || a.type == HA_GEMVT) {
            // Zs[t] = A1[:, t]^T X[i0:i0+ni] (LR) or X[o0 + t] -= A1[:, t]^T X[i0:i0+ni] (GEMVT)
            const T* A1 = (const T*)a.A1;
            const int K = a.type == HA_LR ? a.K : a.no;
            for (int t0 = 0; t0 < K; t0 += HS_ZROWS) {
                const int kt = min(HS_ZROWS, K - t0);
                for (int t = warp; t < kt; t += (int)(blockDim.x >> 5)) {
                    T acc[CW];
#pragma unroll
                    for (int q = 0; q < CW; ++q) acc[q] = T(0);
                    const T* col = A1 + (size_t)(t0 + t) * a.lda1;
#pragma unroll 4
                    for (int i = lane; i < a.ni; i += 32) {
                        const T v = col[i];
#pragma unroll
                        for (int q = 0; q < CW; ++q) acc[q] = fma(v, Xs[(size_t)(a.i0 + i) * CW + q], acc[q]);
                    }
#pragma unroll
                    for (int q = 0; q < CW; ++q) {
                        T v = acc[q];
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                        acc[q] = v;
                    }
                    if (lane == 0) {
#pragma unroll
                        for (int q = 0; q < CW; ++q) {
                            if (a.type == HA_LR) Zs[(size_t)t * CW + q] = acc[q];
                            else Xs[(size_t)(a.o0 + t0 + t) * CW + q] -= acc[q];
                        }
                    }
                }
                __syncthreads();
                if (a.type == HA_LR) {
                    // X[o0:o0+no] -= A2[:, t0:t0+kt] Zs
                    const T* A2 = (const T*)a.A2;
                    for (int i = tid; i < a.no; i += blockDim.x) {
                        T acc[CW];
#pragma unroll
                        for (int q = 0; q < CW; ++q) acc[q] = T(0);
#pragma unroll 8
                        for (int t = 0; t < kt; ++t) {
                            const T v = A2[i + (size_t)(t0 + t) * a.lda2];
#pragma unroll
                            for (int q = 0; q < CW; ++q) acc[q] = fma(v, Zs[(size_t)t * CW + q], acc[q]);
                        }
#pragma unroll
                        for (int q = 0; q < CW; ++q) Xs[(size_t)(a.o0 + i) * CW + q] -= acc[q];
                    }
                    __syncthreads();
                }
            }
        } else {   // HA_GEMV: X[o0:o0+no] -= A2 X[i0:i0+K]
            const T* A2 = (const T*)a.A2;
            for (int i = tid; i < a.no; i += blockDim.x) {
                T acc[CW];
#pragma unroll
                for (int q = 0; q < CW; ++q) acc[q] = T(0);
#pragma unroll 8
                for (int t = 0; t < a.K; ++t) {
                    const T v = A2[i + (size_t)t * a.lda2];
#pragma unroll
                    for (int q = 0; q < CW; ++q) acc[q] = fma(v, Xs[(size_t)(a.i0 + t) * CW + q], acc[q]);
                }
#pragma unroll
                for (int q = 0; q < CW; ++q) Xs[(size_t)(a.o0 + i) * CW + q] -= acc[q];
            }
            __syncthreads();
        }
    }
    for (int e = tid; e < tk.c * CW; e += blockDim.x) {
        const int i = e / CW, q = e % CW;
        if (q < nc) X[(size_t)i * tk.ldx + c0 + q] = Xs[e];
    }
}

// ------------------------------------------------------------------ random test matrices
// Philox4x32-10 (Salmon et al., SC'11): ten rounds, key bumped between rounds.
__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint32_t hi0 = __umulhi(0xD2511F53u, c[0]), lo0 = 0xD2511F53u * c[0];
        uint32_t hi1 = __umulhi(0xCD9E8D57u, c[2]), lo1 = 0xCD9E8D57u * c[2];
        uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
    }
}

// G (m x 16 at columns col0.., row-major, ld): entry (i, c) from counter (i, c/2, block_id, word3), key = seed;
// Box-Muller on (w0, w1) for even c and (w2, w3) for odd c.  32 rows per CTA.
// Two standard normal samples of row i, column pair cp of one sample block: Philox4x32-10 on
// the counter (i, cp, block id, word3), key = seed, then Box-Muller on the two word pairs.
template <class T>
__device__ __forceinline__ void gauss_pair(uint32_t i, uint32_t cp, uint32_t block_id, uint32_t word3,
                                           unsigned long long seed, T& z0, T& z1) {
    uint32_t c[4] = {i, cp, block_id, word3};
    philox4x32_10(c, (uint32_t)(seed & 0xffffffffull), (uint32_t)(seed >> 32));
    if (sizeof(T) == 8) {
        const double two32 = 2.3283064365386963e-10;   // 2^-32
        const double twopi = 6.283185307179586;
        z0 = (T)(sqrt(-2.0 * log(((double)c[0] + 1.0) * two32)) * cos(twopi * ((double)c[1] * two32)));
        z1 = (T)(sqrt(-2.0 * log(((double)c[2] + 1.0) * two32)) * cos(twopi * ((double)c[3] * two32)));
    } else {   // FP32 form: single-precision transforms of the same Philox words
        const float f32 = 2.3283064365386963e-10f, tp = 6.2831853071795865f;
        z0 = (T)(sqrtf(-2.0f * logf(((float)c[0] + 1.0f) * f32)) * cosf(tp * ((float)c[1] * f32)));
        z1 = (T)(sqrtf(-2.0f * logf(((float)c[2] + 1.0f) * f32)) * cosf(tp * ((float)c[3] * f32)));
    }
}

template <class T>
__global__ void k_gauss(const GaussTask* __restrict__ tasks, unsigned long long seed) {
    const GaussTask tk = tasks[blockIdx.x];
    const int i = tk.row0 + (threadIdx.x >> 3), cp = threadIdx.x & 7;
    if (i >= tk.m) return;
    T z0, z1;
    gauss_pair<T>((uint32_t)i, (uint32_t)cp, tk.block_id, tk.word3, seed, z0, z1);
    T* G = (T*)tk.G;
    G[(size_t)i * tk.ld + tk.col0 + 2 * cp] = z0;
    G[(size_t)i * tk.ld + tk.col0 + 2 * cp + 1] = z1;
}

// dst[i*dsr + c*dsc] = src[i*ssr + c*ssc] (or -= with sub); grid (tasks, 32).
template <class T>
__global__ void k_copy(const CopyTask* __restrict__ tasks) {
    const CopyTask tk = tasks[blockIdx.x];
    const long long cnt = (long long)tk.m * tk.nc;
    for (long long e = blockIdx.y * (long long)blockDim.x + threadIdx.x; e < cnt; e += (long long)gridDim.y * blockDim.x) {
        const long long i = tk.nc == 1 ? e : e % tk.m, c = tk.nc == 1 ? 0 : e / tk.m;
        const T v = ((const T*)tk.src)[i * tk.ssr + c * tk.ssc];
        if (tk.sub) ((T*)tk.dst)[i * tk.dsr + c * tk.dsc] -= v;
        else ((T*)tk.dst)[i * tk.dsr + c * tk.dsc] = v;
    }
}

// Row-major thin block <-> strided copies and scaled adds (vector path of the solve).
template <class T>
__global__ void k_axpy_rows(const T* __restrict__ X, int ldx, T* __restrict__ Y, int ldy, int m, int nc, T alpha) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m * nc; e += gridDim.x * blockDim.x) {
        int i = e / nc, c = e % nc;
        Y[(size_t)i * ldy + c] += alpha * X[(size_t)i * ldx + c];
    }
}

template <class T>
__global__ void k_fill(T* __restrict__ X, long long cnt, T v) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < cnt; e += (long long)gridDim.x * blockDim.x)
        X[e] = v;
}

// ------------------------------------------------------------------ permutation and PCG vectors (FP64)
template <class T>
__global__ void k_perm_in(const double* __restrict__ r, const int32_t* __restrict__ perm, T* __restrict__ y, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = (T)r[perm[i]];
}
template <class T>
__global__ void k_perm_out(const T* __restrict__ y, const int32_t* __restrict__ perm, double* __restrict__ z, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        z[perm[i]] = (double)y[i];
}

// X (c x c, row-major) <- identity
template <class T>
__global__ void k_set_identity(T* __restrict__ X, int c) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)c * c;
         e += (long long)gridDim.x * blockDim.x)
        X[e] = (e / c == e % c) ? T(1) : T(0);
}

// N right-hand sides: column c of r / z at offset c n, y row-major (n x N)
template <class T>
__global__ void k_perm_in_cols(const double* __restrict__ r, const int32_t* __restrict__ perm, T* __restrict__ y,
                               long long n, int N) {
    const int c = blockIdx.y;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i * N + c] = (T)r[(size_t)c * n + perm[i]];
}
template <class T>
__global__ void k_perm_out_cols(const T* __restrict__ y, const int32_t* __restrict__ perm, double* __restrict__ z,
                                long long n, int N) {
    const int c = blockIdx.y;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        z[(size_t)c * n + perm[i]] = (double)y[i * N + c];
}

}  // namespace rsc
