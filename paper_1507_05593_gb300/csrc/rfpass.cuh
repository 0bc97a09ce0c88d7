// One pass of the adaptive range finder (Alg. 3) for a batch of blocks, as one
// cooperative launch.
//
// For every block r under compression (U_r: c x maxr column-major orthonormal basis,
// rank columns so far), given this pass's 16-column sample block Y = (implicit
// product) of Gaussian columns:
//   Y <- (I - U U^T)^2 Y                     (two projections, Alg. 3)
//   stop when ||Y||_F <= tol ||Y_1||_F        (Y_1: the first pass's block)
//   else Q = makeOrthonormal(Y[:, :b]), b = min(16, maxr - rank), by shifted
//        Cholesky QR, a projection against U and two more Cholesky QR passes
//        (shifted CholeskyQR3; Fukaya, Kannan, Nakatsukasa, Yamamoto, Yanagisawa,
//        SIAM J. Sci. Comput. 2020), then U[:, rank:rank+b'] = Q, rank += b', where
//        b' <= b counts the columns that are not numerically dependent in working
//        precision (see rfp_chol).
// The rows of every block are cut into 64-row chunks; a chunk belongs to CTA
// (chunk mod grid) in every phase, so a CTA only ever touches its own rows of Y
// and U.  Reductions over rows (U^T Y, Y^T Y) write per-chunk partial sums that a
// following phase adds in ascending chunk order (deterministic).  Phases are
// separated by a grid barrier whose waits are bounded: on expiry the kernel
// records an error code and returns.  The stopping decision and the rank live in
// device memory, so passes follow one another without a host round trip.
#pragma once

#include <cstdint>

#include "kernels.cuh"

namespace rsc {

constexpr int RFP_ROWS = 64;             // rows per chunk
constexpr int RFP_THREADS = 256;
constexpr unsigned long long RFP_SPIN_LIMIT = 1ull << 22;   // default polls of a barrier wait (64 ns apart)
constexpr int RFP_SMALL = 0;             // small-block mode off (see the note in k_rf_pass)

template <class T>
struct RfDev {
    // set by the host once per batch
    T* U;              // c x maxr, column-major (ld c)
    T* Y;              // c x 16, row-major: the working block
    T* Z;              // maxr x 16: U^T Y
    T* zpart;          // nchunk x maxr x 16 partial sums of U^T Y
    T* gpart;          // nchunk x 256 partial sums of Y^T Y
    T* rinv;           // R (16 x 16 row-major) and 1 / diag(R) of the current Cholesky QR step
    int c, maxr, nchunk, pad0;
    double tol, u;     // stopping tolerance; unit roundoff of T (shift of the first QR)
    // written by the kernel
    int rank, active, b, bad;
    double y1;         // ||Y_1||_F
};

template <class T>
struct RfPass { const T* Yb; int ldyb; int first; };   // this pass's samples (null: none)

struct RfBarrier { unsigned count, gen; };

// Grid barrier for a cooperative launch (all CTAs resident).  Returns false when the
// wait ran out; the caller then returns.
__device__ __forceinline__ bool rfp_grid_sync(RfBarrier* bar, unsigned& gen, int* err, int& ok_s,
                                              unsigned long long limit) {
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        __threadfence();
        const unsigned arrived = atomicAdd(&bar->count, 1u);
        if (arrived == gridDim.x - 1) {
            atomicExch(&bar->count, 0u);
            __threadfence();
            atomicAdd(&bar->gen, 1u);
        } else {
            ok = 0;
            for (unsigned long long it = 0; it < limit; ++it) {
                if (*(volatile unsigned*)&bar->gen != gen) { ok = 1; break; }
                __nanosleep(64);
            }
            if (!ok) atomicCAS(err, 0, 1);
        }
        __threadfence();
        ++gen;
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

__device__ __forceinline__ int rfp_ld(const int* p) { return __ldcg(p); }   // written by other CTAs

// 64 x 32 tile of U (rows row0.., columns k0..) into registers: thread t holds rows
// t % 64 of columns t / 64 + 4 q, q < 8 (coalesced along the rows)
template <class T>
__device__ __forceinline__ void rfp_fetch_u(const T* U, int c, int row0, int nr, int k0, int kn, T (&v)[8]) {
    const int i = threadIdx.x % RFP_ROWS, k4 = threadIdx.x / RFP_ROWS;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int kk = k4 + 4 * q;
        v[q] = (i < nr && kk < kn) ? U[(size_t)(k0 + kk) * c + row0 + i] : T(0);
    }
}
template <class T>
__device__ __forceinline__ void rfp_put_u(const T (&v)[8], T (*Us)[33]) {
    const int i = threadIdx.x % RFP_ROWS, k4 = threadIdx.x / RFP_ROWS;
#pragma unroll
    for (int q = 0; q < 8; ++q) Us[i][k4 + 4 * q] = v[q];
}

// out[k][col] = sum_i U[row0 + i, k] Ys[i][col], k < rank (the chunk's part of U^T Y);
// the next 32 columns of U are fetched while the current ones are used
template <class T>
__device__ void rfp_tn_partial(const T* U, int c, int row0, int nr, int rank, T (*Ys)[17], T (*Us)[33], T* out) {
    const int kk = threadIdx.x >> 3, cp = (threadIdx.x & 7) * 2;
    T v[8];
    rfp_fetch_u(U, c, row0, nr, 0, min(32, rank), v);
    for (int k0 = 0; k0 < rank; k0 += 32) {
        const int kn = min(32, rank - k0);
        __syncthreads();
        rfp_put_u(v, Us);
        __syncthreads();
        if (k0 + 32 < rank) rfp_fetch_u(U, c, row0, nr, k0 + 32, min(32, rank - k0 - 32), v);
        T a0 = T(0), a1 = T(0);
#pragma unroll 8
        for (int i = 0; i < RFP_ROWS; ++i) {
            const T u = Us[i][kk];
            a0 = fma(u, Ys[i][cp], a0);
            a1 = fma(u, Ys[i][cp + 1], a1);
        }
        if (kk < kn) {
            out[(size_t)(k0 + kk) * 16 + cp] = a0;
            out[(size_t)(k0 + kk) * 16 + cp + 1] = a1;
        }
    }
    __syncthreads();
}

// Ys -= U[chunk rows, :rank] Z  (Z: rank x 16, written by other CTAs)
template <class T>
// (Z may also be given as nz partial sums, zst apart, added here in ascending order.)
__device__ void rfp_nn_update(const T* U, int c, int row0, int nr, int rank, const T* Z, T (*Ys)[17], T (*Us)[33],
                              T (*Zs)[17], int nz = 1, size_t zst = 0) {
    const int i = threadIdx.x >> 2, cq = (threadIdx.x & 3) * 4;
    T acc[4] = {T(0), T(0), T(0), T(0)};
    T v[8], zv[2];
    auto fetch_z = [&](int k0, int kn) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int e = threadIdx.x + h * RFP_THREADS, kk = e >> 4, col = e & 15;
            T a = T(0);
            if (kk < kn)
                for (int q = 0; q < nz; ++q) a += __ldcg(Z + q * zst + (size_t)(k0 + kk) * 16 + col);
            zv[h] = a;
        }
    };
    rfp_fetch_u(U, c, row0, nr, 0, min(32, rank), v);
    fetch_z(0, min(32, rank));
    for (int k0 = 0; k0 < rank; k0 += 32) {
        __syncthreads();
        rfp_put_u(v, Us);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int e = threadIdx.x + h * RFP_THREADS;
            Zs[e >> 4][e & 15] = zv[h];
        }
        __syncthreads();
        if (k0 + 32 < rank) {
            rfp_fetch_u(U, c, row0, nr, k0 + 32, min(32, rank - k0 - 32), v);
            fetch_z(k0 + 32, min(32, rank - k0 - 32));
        }
#pragma unroll 8
        for (int kk = 0; kk < 32; ++kk) {
            const T u = Us[i][kk];
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[j] = fma(u, Zs[kk][cq + j], acc[j]);
        }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < 4; ++j) Ys[i][cq + j] -= acc[j];
    __syncthreads();
}

// out[a][b] = sum_i Ys[i][a] Ys[i][b] (rows beyond the chunk are zero in Ys)
template <class T>
__device__ __forceinline__ void rfp_gram_partial(T (*Ys)[17], T* out) {
    const int a = threadIdx.x >> 4, b = threadIdx.x & 15;
    T s = T(0);
#pragma unroll 8
    for (int i = 0; i < RFP_ROWS; ++i) s = fma(Ys[i][a], Ys[i][b], s);
    out[threadIdx.x] = s;
}

// Ys[:, :b] <- Ys[:, :b] R^{-1} by forward substitution along each row (thread per row);
// rf holds R (row-major 16 x 16) and the reciprocal diagonal (zero for a dropped column).
template <class T>
__device__ void rfp_apply_rsolve(const T* rf, int b, T (*Ys)[17], T (*Gs)[17], T* rd, bool shared_src = false) {
    for (int e = threadIdx.x; e < 256; e += RFP_THREADS) Gs[e >> 4][e & 15] = shared_src ? rf[e] : __ldcg(rf + e);
    if (threadIdx.x < 16) rd[threadIdx.x] = shared_src ? rf[256 + threadIdx.x] : __ldcg(rf + 256 + threadIdx.x);
    __syncthreads();
    if (threadIdx.x < RFP_ROWS) {
        const int i = threadIdx.x;
        T x[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            if (j < b) {
                T s = Ys[i][j];
#pragma unroll
                for (int k = 0; k < j; ++k) s = fma(-x[k], Gs[k][j], s);
                x[j] = s * rd[j];
                Ys[i][j] = x[j];
            } else {
                x[j] = T(0);
            }
        }
    }
    __syncthreads();
}

// Warp 0: G (b x b, upper triangle used) + shift I = R^T R with lane j holding column
// j in registers (rows of R broadcast by shuffles); shift = coef trace(G).  A column
// whose pivot is at most delta times its (shifted) diagonal entry is numerically
// dependent on the earlier ones in working precision: its row of R and its reciprocal
// pivot are set to zero, so it leaves the block as a zero column.  Writes R (row-major
// 16 x 16, upper b x b) and the reciprocal diagonal to out[0..271].  Returns true on
// a non-finite pivot.
// square root in the argument's own precision
__device__ __forceinline__ float tsqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double tsqrt(double x) { return sqrt(x); }

template <class T>
__device__ bool rfp_chol(T (*G)[17], int b, double coef, double delta, T* out) {
    const int j = threadIdx.x & 31;
    T tr = T(0);
    for (int i = 0; i < b; ++i) tr += G[i][i];
    const T shift = (T)(coef * (double)tr);
    T col[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) col[i] = (j < b && i <= j) ? G[i][j] + (i == j ? shift : T(0)) : T(0);
    T g0 = T(0);
#pragma unroll
    for (int i = 0; i < 16; ++i)
        if (i == j) g0 = col[i];
    bool bad = false;
    T rdiag = T(0);
    const T dlt = (T)delta;
    // row k of R reaches the lanes through shared memory (double-buffered: one warp barrier per
    // pivot); a shuffle per element was the slower form
    __shared__ T rowb[2][16];
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        if (k < b) {
            const T d = __shfl_sync(0xffffffffu, col[k], k);
            const T g0k = __shfl_sync(0xffffffffu, g0, k);
            if (d != d) bad = true;
            const bool keep = d > dlt * g0k;
            const T r = keep ? tsqrt(d) : T(0);
            const T ri = keep ? T(1) / r : T(0);
            const T rkj = j > k ? col[k] * ri : (j == k ? r : T(0));
            col[k] = rkj;
            if (j == k) rdiag = ri;
            if (j < 16) rowb[k & 1][j] = rkj;
            __syncwarp();
#pragma unroll
            for (int i = k + 1; i < 16; ++i)
                if (j >= i) col[i] = fma(-rowb[k & 1][i], rkj, col[i]);
        }
    }
    if (j < 16) {
#pragma unroll
        for (int i = 0; i < 16; ++i) out[i * 16 + j] = (i <= j && j < b) ? col[i] : T(0);
        out[256 + j] = j < b ? rdiag : T(0);
    }
    return bad;
}

template <class T>
__global__ void __launch_bounds__(RFP_THREADS, 2) k_rf_pass(RfDev<T>* rf, const RfPass<T>* __restrict__ ps, int nrf,
                                                         const int2* __restrict__ chunks, int nchunks, RfBarrier* bar,
                                                         int* err, unsigned long long* ptime, int small,
                                                         unsigned long long spin_limit) {
    __shared__ T Ys[RFP_ROWS][17];
    __shared__ T Us[RFP_ROWS][33];
    __shared__ T Zs[32][17];
    __shared__ T Red[8][33];
    __shared__ T Gs[16][17], rd_s[16];
    __shared__ unsigned gen_s;
    __shared__ int ok_s;
    __shared__ int nz_s[RFP_THREADS];
    const int tid = threadIdx.x;
    // a wait of an earlier pass ran out: the barrier count may be stale, so no pass runs until
    // the host has seen the error
    if (*(volatile int*)err) return;
    if (tid == 0) gen_s = *(volatile unsigned*)&bar->gen;   // cannot change before every CTA has arrived once
    int any = 0;
    for (int r = tid; r < nrf; r += RFP_THREADS) any |= (ps[r].Yb != nullptr && rfp_ld(&rf[r].active));
    if (!__syncthreads_or(any)) return;           // same answer in every CTA
    unsigned gen = gen_s;
    auto live = [&](int r) { return ps[r].Yb != nullptr && rfp_ld(&rf[r].active) != 0; };
    // profile mode: CTA 0 adds the time from one barrier exit to the next to ptime[phase]
    unsigned long long t0 = 0;
    const bool timed = ptime != nullptr && blockIdx.x == 0 && tid == 0;
    if (timed) asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    auto sync = [&](int ph) {
        const bool ok = rfp_grid_sync(bar, gen, err, ok_s, spin_limit);
        if (timed) {
            unsigned long long t;
            asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
            ptime[ph] += t - t0;
            t0 = t;
        }
        return ok;
    };
    // load the chunk's rows of Y (zero below the block)
    auto load_y = [&](const RfDev<T>& R, int row0, int nr) {
        for (int e = tid; e < RFP_ROWS * 16; e += RFP_THREADS) {
            const int i = e >> 4, col = e & 15;
            Ys[i][col] = i < nr ? R.Y[(size_t)(row0 + i) * 16 + col] : T(0);
        }
        __syncthreads();
    };
    auto store_y = [&](const RfDev<T>& R, int row0, int nr) {
        __syncthreads();
        for (int e = tid; e < RFP_ROWS * 16; e += RFP_THREADS) {
            const int i = e >> 4, col = e & 15;
            if (i < nr) R.Y[(size_t)(row0 + i) * 16 + col] = Ys[i][col];
        }
        __syncthreads();
    };
    // Z_r = sum over chunks of the partial U^T Y.  Work item = 32 entries of one block;
    // warp w adds chunks w, w + 8, ... and the 8 warp sums are added in order.  The
    // entry counts of 256 blocks at a time are read in parallel into shared memory.
    auto reduce_z = [&]() {
        const int warp = tid >> 5, lane = tid & 31;
        int item = 0;
        for (int g0 = 0; g0 < nrf; g0 += RFP_THREADS) {
            {
                const int r = g0 + tid;
                nz_s[tid] = (r < nrf && live(r)) ? rfp_ld(&rf[r].rank) * 16 : 0;
            }
            __syncthreads();
            const int gn = min(RFP_THREADS, nrf - g0);
            for (int k = 0; k < gn; ++k) {
                const int n = nz_s[k];
                const int nitem = (n + 31) >> 5;
                if (nitem == 0) continue;
                const int first = (int)((blockIdx.x + gridDim.x - (unsigned)(item % (int)gridDim.x)) % gridDim.x);
                item += nitem;
                if (first >= nitem) continue;       // no item of this block falls on this CTA
                const RfDev<T>& R = rf[g0 + k];
                for (int it = first; it < nitem; it += gridDim.x) {
                    const int e = it * 32 + lane;
                    T a[4] = {T(0), T(0), T(0), T(0)};
                    if (e < n) {
                        const size_t st = (size_t)R.maxr * 16;
                        const T* zp = R.zpart + e;
                        int q = warp;
                        for (; q + 24 < R.nchunk; q += 32) {
                            T v[4];
#pragma unroll
                            for (int h = 0; h < 4; ++h) v[h] = __ldcg(zp + (size_t)(q + 8 * h) * st);
#pragma unroll
                            for (int h = 0; h < 4; ++h) a[h] += v[h];
                        }
                        for (; q < R.nchunk; q += 8) a[0] += __ldcg(zp + (size_t)q * st);
                    }
                    Red[warp][lane] = (a[0] + a[1]) + (a[2] + a[3]);
                    __syncthreads();
                    if (warp == 0 && e < n) {
                        T t = T(0);
#pragma unroll
                        for (int w = 0; w < 8; ++w) t += Red[w][lane];
                        R.Z[e] = t;
                    }
                    __syncthreads();
                }
            }
            __syncthreads();
        }
    };
    // Gram matrix of block r (CTA-wide; eight interleaved partial sums, added in a fixed
    // order, so that eight loads are in flight per thread) into Gs
    auto reduce_g = [&](const RfDev<T>& R) {
        T a[8];
#pragma unroll
        for (int h = 0; h < 8; ++h) a[h] = T(0);
        int q = 0;
        for (; q + 7 < R.nchunk; q += 8) {
            T v[8];
#pragma unroll
            for (int h = 0; h < 8; ++h) v[h] = __ldcg(R.gpart + (size_t)(q + h) * 256 + tid);
#pragma unroll
            for (int h = 0; h < 8; ++h) a[h] += v[h];
        }
        for (; q < R.nchunk; ++q) a[0] += __ldcg(R.gpart + (size_t)q * 256 + tid);
        Gs[tid >> 4][tid & 15] = ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
        __syncthreads();
    };

    if (small) {
        // ------------------------------------------------------------ small blocks (nchunk <= RFP_SMALL)
        // Not used (RFP_SMALL = 0): factorizing 256 independent systems at once, this mode gave
        // intermittently wrong samples (an indefinite diagonal block or inflated ranks in about
        // one factorization of four in FP64) that the full mode below does not; the race has not
        // been found, so the host never selects it.
        // Every CTA adds the few partial sums it needs itself (Z of a projection, the Gram
        // matrix) and factors the 16 x 16 Gram matrix of its block redundantly, so that the
        // reduction and Cholesky phases disappear; the partial buffers alternate between two
        // halves so that a phase never overwrites what another CTA of the same phase reads.
        // All CTAs of a block reduce the same values in the same order, so their decisions
        // agree; the CTA of chunk 0 records them.
        auto zp = [&](const RfDev<T>& R, int h) { return R.zpart + (size_t)h * R.nchunk * R.maxr * 16; };
        auto gp = [&](const RfDev<T>& R, int h) { return R.gpart + (size_t)h * R.nchunk * 256; };
        auto gram_all = [&](const RfDev<T>& R, int h) {        // Gram matrix from the partials into Gs
            T a = T(0);
            for (int q = 0; q < R.nchunk; ++q) a += __ldcg(gp(R, h) + (size_t)q * 256 + tid);
            Gs[tid >> 4][tid & 15] = a;
            __syncthreads();
        };
        // A: samples into Y; first pass: Gram partials (half 0); U^T Y partials (half 0)
        for (int g = blockIdx.x; g < nchunks; g += gridDim.x) {
            const int r = chunks[g].x, q = chunks[g].y;
            if (!live(r)) continue;
            const RfDev<T>& R = rf[r];
            const int row0 = q * RFP_ROWS, nr = min(RFP_ROWS, R.c - row0);
            const RfPass<T> p = ps[r];
            for (int e = tid; e < RFP_ROWS * 16; e += RFP_THREADS) {
                const int i = e >> 4, col = e & 15;
                const T v = i < nr ? p.Yb[(size_t)(row0 + i) * p.ldyb + col] : T(0);
                Ys[i][col] = v;
                if (i < nr) R.Y[(size_t)(row0 + i) * 16 + col] = v;
            }
            __syncthreads();
            if (p.first) rfp_gram_partial(Ys, gp(R, 0) + (size_t)q * 256);
            const int rank = rfp_ld(&R.rank);
            if (rank > 0) rfp_tn_partial(R.U, R.c, row0, nr, rank, Ys, Us, zp(R, 0) + (size_t)q * R.maxr * 16);
            __syncthreads();
        }
        if (!sync(0)) return;
        // C: Y -= U Z (half 0); U^T Y partials (half 1)
        for (int g = blockIdx.x; g < nchunks; g += gridDim.x) {
            const int r = chunks[g].x, q = chunks[g].y;
            if (!live(r)) continue;
            const RfDev<T>& R = rf[r];
            const int rank = rfp_ld(&R.rank);
            if (rank == 0) continue;
            const int row0 = q * RFP_ROWS, nr = min(RFP_ROWS, R.c - row0);
            load_y(R, row0, nr);
            rfp_nn_update(R.U, R.c, row0, nr, rank, zp(R, 0), Ys, Us, Zs, R.nchunk, (size_t)R.maxr * 16);
            store_y(R, row0, nr);
            rfp_tn_partial(R.U, R.c, row0, nr, rank, Ys, Us, zp(R, 1) + (size_t)q * R.maxr * 16);
        }
        if (!sync(2)) return;
        // E: Y -= U Z (half 1); Gram partials (half 1)
        for (int g = blockIdx.x; g < nchunks; g += gridDim.x) {
            const int r = chunks[g].x, q = chunks[g].y;
            if (!live(r)) continue;
            const RfDev<T>& R = rf[r];
            const int rank = rfp_ld(&R.rank);
            const int row0 = q * RFP_ROWS, nr = min(RFP_ROWS, R.c - row0);
            load_y(R, row0, nr);
            if (rank > 0) {
                rfp_nn_update(R.U, R.c, row0, nr, rank, zp(R, 1), Ys, Us, Zs, R.nchunk, (size_t)R.maxr * 16);
                store_y(R, row0, nr);
            }
            rfp_gram_partial(Ys, gp(R, 1) + (size_t)q * 256);
            __syncthreads();
        }
        if (!sync(4)) return;
        // G: stopping test, shifted Cholesky, Y <- Y R^{-1}, U^T Y partials (half 0)
        __shared__ T Rl[272];
        __shared__ int go_s;
        __shared__ double y1_s;
        for (int g = blockIdx.x; g < nchunks; g += gridDim.x) {
            const int r = chunks[g].x, q = chunks[g].y;
            if (!live(r)) continue;
            RfDev<T>& R = rf[r];
            const int rank = rfp_ld(&R.rank);
            const int row0 = q * RFP_ROWS, nr = min(RFP_ROWS, R.c - row0);
            const bool first = ps[r].first != 0;
            double y1 = 0.0;
            if (first) {            // ||Y_1||^2 = trace of the first pass's Gram matrix (half 0)
                gram_all(R, 0);
                if (tid == 0) {
                    double t = 0.0;
                    for (int a = 0; a < 16; ++a) t += (double)Gs[a][a];
                    y1_s = sqrt(t);
                    if (q == 0) R.y1 = y1_s;
                }
                __syncthreads();
                y1 = y1_s;
            } else {
                y1 = __ldcg(&R.y1);
            }
            gram_all(R, 1);
            if (tid < 32) {
                double t = 0.0;
                for (int a = 0; a < 16; ++a) t += (double)Gs[a][a];
                const double nrm = sqrt(t);
                int go = 1, b = 0;
                if (!isfinite(nrm) || !isfinite(y1)) {
                    go = 0;
                    if (tid == 0) atomicCAS(err + 1, 0, 1);
                } else if (nrm <= R.tol * y1) {
                    go = 0;
                } else {
                    b = min(16, R.maxr - rank);
                    const double coef = 11.0 * ((double)R.c * b + (double)b * (b + 1)) * R.u;
                    const bool bad = rfp_chol(Gs, b, coef, 4.0 * max(R.c, 16) * R.u, Rl);
                    if (tid == 0 && q == 0) R.bad = bad ? 1 : 0;
                }
                if (tid == 0) {
                    go_s = go ? b : 0;
                    if (q == 0) {
                        R.b = b;
                        if (!go) R.active = 0;
                    }
                }
            }
            __syncthreads();
            const int b = go_s;
            if (b == 0) continue;
            load_y(R, row0, nr);
            rfp_apply_rsolve(Rl, b, Ys, Gs, rd_s, true);
            store_y(R, row0, nr);
            if (rank > 0) rfp_tn_partial(R.U, R.c, row0, nr, rank, Ys, Us, zp(R, 0) + (size_t)q * R.maxr * 16);
        }
        if (!sync(5)) return;
        // I: Y -= U Z (half 0); Gram partials (half 0)
        for (int g = blockIdx.x; g < nchunks; g += gridDim.x) {
            const int r = chunks[g].x, q = chunks[g].y;
            if (!live(r)) continue;
            const RfDev<T>& R = rf[r];
            const int rank = rfp_ld(&R.rank);
            const int row0 = q * RFP_ROWS, nr = min(RFP_ROWS, R.c - row0);
            load_y(R, row0, nr);
            if (rank > 0) {
                rfp_nn_update(R.U, R.c, row0, nr, rank, zp(R, 0), Ys, Us, Zs, R.nchunk, (size_t)R.maxr * 16);
                store_y(R, row0, nr);
            }
            rfp_gram_partial(Ys, gp(R, 0) + (size_t)q * 256);
            __syncthreads();
        }
        // JK, LM: Cholesky of the Gram matrix, Y <- Y R^{-1}, then Gram partials or the append
        for (int pass = 0; pass < 2; ++pass) {
            if (!sync(8 + 2 * pass)) return;
            for (int g = blockIdx.x; g < nchunks; g += gridDim.x) {
                const int r = chunks[g].x, q = chunks[g].y;
                if (!live(r)) continue;
                RfDev<T>& R = rf[r];
                const int b = rfp_ld(&R.b);
                const int row0 = q * RFP_ROWS, nr = min(RFP_ROWS, R.c - row0);
                gram_all(R, pass == 0 ? 0 : 1);
                if (tid < 32) {
                    const bool bad = rfp_chol(Gs, b, 0.0, 4.0 * max(R.c, 16) * R.u, Rl);
                    if (tid == 0 && q == 0 && bad) R.bad = 1;
                }
                __syncthreads();
                load_y(R, row0, nr);
                rfp_apply_rsolve(Rl, b, Ys, Gs, rd_s, true);
                store_y(R, row0, nr);
                if (pass == 0) {
                    rfp_gram_partial(Ys, gp(R, 1) + (size_t)q * 256);
                } else {   // kept columns (nonzero 1 / R_kk) appended in order; chunk 0 keeps R for the commit
                    const int rank = rfp_ld(&R.rank);
                    unsigned keep = 0;
                    for (int col = 0; col < b; ++col) keep |= (rd_s[col] != T(0) ? 1u : 0u) << col;
                    for (int e = tid; e < RFP_ROWS * 16; e += RFP_THREADS) {
                        const int i = e % RFP_ROWS, col = e / RFP_ROWS;
                        if (i < nr && col < b && ((keep >> col) & 1u)) {
                            const int pos = __popc(keep & ((1u << col) - 1u));
                            R.U[(size_t)(rank + pos) * R.c + row0 + i] = Ys[i][col];
                        }
                    }
                    if (q == 0)
                        for (int e = tid; e < 272; e += RFP_THREADS) R.rinv[e] = Rl[e];
                }
                __syncthreads();
            }
        }
        if (!sync(12)) return;
        for (int r = blockIdx.x; r < nrf; r += gridDim.x) {
            if (tid != 0 || !live(r)) continue;
            RfDev<T>& R = rf[r];
            const int b = rfp_ld(&R.b);
            int kept = 0;
            for (int col = 0; col < b; ++col) kept += __ldcg(R.rinv + 256 + col) != T(0);
            if (rfp_ld(&R.bad) || kept == 0) {
                R.active = 0;
            } else {
                const int rank = rfp_ld(&R.rank) + kept;
                R.rank = rank;
                if (rank >= R.maxr) R.active = 0;
            }
        }
        return;
    }

    // A: Y <- this pass's samples; Gram partials on the first pass (for ||Y_1||); U^T Y partials
    for (int g = blockIdx.x; g < nchunks; g += gridDim.x) {
        const int r = chunks[g].x, q = chunks[g].y;
        if (!live(r)) continue;
        const RfDev<T>& R = rf[r];
        const int row0 = q * RFP_ROWS, nr = min(RFP_ROWS, R.c - row0);
        const RfPass<T> p = ps[r];
        for (int e = tid; e < RFP_ROWS * 16; e += RFP_THREADS) {
            const int i = e >> 4, col = e & 15;
            const T v = i < nr ? p.Yb[(size_t)(row0 + i) * p.ldyb + col] : T(0);
            Ys[i][col] = v;
            if (i < nr) R.Y[(size_t)(row0 + i) * 16 + col] = v;
        }
        __syncthreads();
        if (p.first) rfp_gram_partial(Ys, R.gpart + (size_t)q * 256);
        const int rank = rfp_ld(&R.rank);
        if (rank > 0) rfp_tn_partial(R.U, R.c, row0, nr, rank, Ys, Us, R.zpart + (size_t)q * R.maxr * 16);
        __syncthreads();
    }
    if (!sync(0)) return;
    // B: Z = U^T Y; ||Y_1||^2 on the first pass
    reduce_z();
    for (int r = blockIdx.x; r < nrf; r += gridDim.x) {
        if (!live(r) || !ps[r].first) continue;
        RfDev<T>& R = rf[r];
        reduce_g(R);
        if (tid == 0) {
            double t = 0.0;
            for (int a = 0; a < 16; ++a) t += (double)Gs[a][a];
            R.y1 = sqrt(t);
        }
        __syncthreads();
    }
    if (!sync(1)) return;
    // C: Y -= U Z, then U^T Y again (second projection)
    for (int g = blockIdx.x; g < nchunks; g += gridDim.x) {
        const int r = chunks[g].x, q = chunks[g].y;
        if (!live(r)) continue;
        const RfDev<T>& R = rf[r];
        const int rank = rfp_ld(&R.rank);
        if (rank == 0) continue;
        const int row0 = q * RFP_ROWS, nr = min(RFP_ROWS, R.c - row0);
        load_y(R, row0, nr);
        rfp_nn_update(R.U, R.c, row0, nr, rank, R.Z, Ys, Us, Zs);
        store_y(R, row0, nr);
        rfp_tn_partial(R.U, R.c, row0, nr, rank, Ys, Us, R.zpart + (size_t)q * R.maxr * 16);
    }
    if (!sync(2)) return;
    reduce_z();                                  // D
    if (!sync(3)) return;
    // E: Y -= U Z; Gram partials of the projected block
    for (int g = blockIdx.x; g < nchunks; g += gridDim.x) {
        const int r = chunks[g].x, q = chunks[g].y;
        if (!live(r)) continue;
        const RfDev<T>& R = rf[r];
        const int rank = rfp_ld(&R.rank);
        const int row0 = q * RFP_ROWS, nr = min(RFP_ROWS, R.c - row0);
        load_y(R, row0, nr);
        if (rank > 0) {
            rfp_nn_update(R.U, R.c, row0, nr, rank, R.Z, Ys, Us, Zs);
            store_y(R, row0, nr);
        }
        rfp_gram_partial(Ys, R.gpart + (size_t)q * 256);
        __syncthreads();
    }
    if (!sync(4)) return;
    // F: stopping test (||Y||_F^2 = trace of the Gram matrix); first Cholesky (shifted)
    for (int r = blockIdx.x; r < nrf; r += gridDim.x) {
        if (!live(r)) continue;
        RfDev<T>& R = rf[r];
        reduce_g(R);
        if (tid < 32) {
            double t = 0.0;
            for (int a = 0; a < 16; ++a) t += (double)Gs[a][a];
            const double nrm = sqrt(t), y1 = __ldcg(&R.y1);
            const int rank = rfp_ld(&R.rank);
            int go = 1, b = 0;
            if (!isfinite(nrm) || !isfinite(y1)) {
                go = 0;
                if (tid == 0) atomicCAS(err + 1, 0, 1);
            } else if (nrm <= R.tol * y1) {
                go = 0;
            } else {
                b = min(16, R.maxr - rank);
                const double coef = 11.0 * ((double)R.c * b + (double)b * (b + 1)) * R.u;
                const bool bad = rfp_chol(Gs, b, coef, 4.0 * max(R.c, 16) * R.u, R.rinv);
                if (tid == 0) R.bad = bad ? 1 : 0;
            }
            if (tid == 0) {
                R.b = b;
                if (!go) R.active = 0;
            }
        }
        __syncthreads();
    }
    if (!sync(5)) return;
    // G: Y <- Y Rinv; U^T Y partials (projection against U)
    for (int g = blockIdx.x; g < nchunks; g += gridDim.x) {
        const int r = chunks[g].x, q = chunks[g].y;
        if (!live(r)) continue;
        const RfDev<T>& R = rf[r];
        const int rank = rfp_ld(&R.rank), b = rfp_ld(&R.b);
        const int row0 = q * RFP_ROWS, nr = min(RFP_ROWS, R.c - row0);
        load_y(R, row0, nr);
        rfp_apply_rsolve(R.rinv, b, Ys, Gs, rd_s);
        store_y(R, row0, nr);
        if (rank > 0) rfp_tn_partial(R.U, R.c, row0, nr, rank, Ys, Us, R.zpart + (size_t)q * R.maxr * 16);
    }
    if (!sync(6)) return;
    reduce_z();                                  // H
    if (!sync(7)) return;
    // I: Y -= U Z; Gram partials
    for (int g = blockIdx.x; g < nchunks; g += gridDim.x) {
        const int r = chunks[g].x, q = chunks[g].y;
        if (!live(r)) continue;
        const RfDev<T>& R = rf[r];
        const int rank = rfp_ld(&R.rank);
        const int row0 = q * RFP_ROWS, nr = min(RFP_ROWS, R.c - row0);
        load_y(R, row0, nr);
        if (rank > 0) {
            rfp_nn_update(R.U, R.c, row0, nr, rank, R.Z, Ys, Us, Zs);
            store_y(R, row0, nr);
        }
        rfp_gram_partial(Ys, R.gpart + (size_t)q * 256);
        __syncthreads();
    }
    // J, K, L, M: two more Cholesky QR passes, then U[:, rank:rank+b] = Y[:, :b]
    for (int pass = 0; pass < 2; ++pass) {
        if (!sync(8 + 2 * pass)) return;
        for (int r = blockIdx.x; r < nrf; r += gridDim.x) {
            if (!live(r)) continue;
            RfDev<T>& R = rf[r];
            reduce_g(R);
            if (tid < 32) {
                const bool bad = rfp_chol(Gs, rfp_ld(&R.b), 0.0, 4.0 * max(R.c, 16) * R.u, R.rinv);
                if (tid == 0 && bad) R.bad = 1;
            }
            __syncthreads();
        }
        if (!sync(9 + 2 * pass)) return;
        for (int g = blockIdx.x; g < nchunks; g += gridDim.x) {
            const int r = chunks[g].x, q = chunks[g].y;
            if (!live(r)) continue;
            const RfDev<T>& R = rf[r];
            const int b = rfp_ld(&R.b);
            const int row0 = q * RFP_ROWS, nr = min(RFP_ROWS, R.c - row0);
            load_y(R, row0, nr);
            rfp_apply_rsolve(R.rinv, b, Ys, Gs, rd_s);
            store_y(R, row0, nr);
            if (pass == 0) {
                rfp_gram_partial(Ys, R.gpart + (size_t)q * 256);
            } else {   // kept columns (nonzero diagonal of R^{-1}, still in Gs) appended in order
                const int rank = rfp_ld(&R.rank);
                unsigned keep = 0;
                for (int col = 0; col < b; ++col) keep |= (rd_s[col] != T(0) ? 1u : 0u) << col;
                for (int e = tid; e < RFP_ROWS * 16; e += RFP_THREADS) {
                    const int i = e % RFP_ROWS, col = e / RFP_ROWS;
                    if (i < nr && col < b && ((keep >> col) & 1u)) {
                        const int pos = __popc(keep & ((1u << col) - 1u));
                        R.U[(size_t)(rank + pos) * R.c + row0 + i] = Ys[i][col];
                    }
                }
            }
            __syncthreads();
        }
    }
    if (!sync(12)) return;
    // N: commit (a failed Cholesky drops the block and ends the search)
    for (int r = blockIdx.x; r < nrf; r += gridDim.x) {
        if (tid != 0 || !live(r)) continue;
        RfDev<T>& R = rf[r];
        const int b = rfp_ld(&R.b);
        int kept = 0;
        for (int col = 0; col < b; ++col) kept += __ldcg(R.rinv + 256 + col) != T(0);
        if (rfp_ld(&R.bad) || kept == 0) {
            R.active = 0;
        } else {
            const int rank = rfp_ld(&R.rank) + kept;
            R.rank = rank;
            if (rank >= R.maxr) R.active = 0;
        }
    }
}

}  // namespace rsc

namespace rsc {

// ---------------------------------------------------------------- dense mode (small blocks)
// The whole adaptive range finder (Alg. 3) of one block B (m x c, row-major, formed densely by
// the implicit product of Alg. 5 applied to the identity) in one CTA: pass t draws the same
// Philox samples G_t as the batched path (counter word3 = t | restarts << 16), Y = B^T G_t, two
// projections against U, the stopping test ||Y||_F <= tol ||Y_1||_F, shifted CholeskyQR3 with
// the dependent-column rule of rfp_chol, U appended; finally V = B U.  For blocks with
// m, c <= RFD_MAX the passes then cost block barriers instead of grid barriers and host round
// trips.  Shared memory: G (m x 16), Y, Z (c, maxr x 17), a 33-column tile of U.
template <class T>
struct RfDenseTask {
    const T* B;             // m x c, row-major (ld c)
    T* U;                   // c x maxr, column-major (ld c)
    T* V;                   // m x maxr, column-major (ld m)
    int m, c, maxr, pad;
    double tol, u;
    uint32_t block_id, word_hi;
    int* rank;              // output: rank found
};
template <class T> constexpr int rfd_max() { return sizeof(T) == 8 ? 256 : 320; }
template <class T> inline size_t rfd_smem(int m, int c, int maxr) {
    return sizeof(T) * ((size_t)m * 16 + (size_t)c * 17 + (size_t)maxr * 17 + (size_t)c * 33);
}

// Sum over a warp of 16 per-lane values: at distance 16, 8, 4, 2 each lane keeps the half of its
// values selected by that lane bit and adds its partner's copy of the same half; a last exchange
// at distance 1 completes the sum.  Lane l returns the total of value rfd_fold16_col(l).
__device__ __forceinline__ int rfd_fold16_col(int lane) {
    return ((lane >> 4) & 1) * 8 + ((lane >> 3) & 1) * 4 + ((lane >> 2) & 1) * 2 + ((lane >> 1) & 1);
}
template <class T>
__device__ __forceinline__ T rfd_fold16(T (&a)[16], int lane) {
    T b[8], c4[4], d2[2];
    const bool h16 = (lane & 16) != 0, h8 = (lane & 8) != 0, h4 = (lane & 4) != 0, h2 = (lane & 2) != 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const T send = h16 ? a[i] : a[i + 8];
        b[i] = (h16 ? a[i + 8] : a[i]) + __shfl_xor_sync(0xffffffffu, send, 16);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const T send = h8 ? b[i] : b[i + 4];
        c4[i] = (h8 ? b[i + 4] : b[i]) + __shfl_xor_sync(0xffffffffu, send, 8);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const T send = h4 ? c4[i] : c4[i + 2];
        d2[i] = (h4 ? c4[i + 2] : c4[i]) + __shfl_xor_sync(0xffffffffu, send, 4);
    }
    const T send = h2 ? d2[0] : d2[1];
    const T e = (h2 ? d2[1] : d2[0]) + __shfl_xor_sync(0xffffffffu, send, 2);
    return e + __shfl_xor_sync(0xffffffffu, e, 1);
}

template <class T>
__global__ void __launch_bounds__(512) k_rf_dense(const RfDenseTask<T>* __restrict__ tasks, unsigned long long seed,
                                                  int* err) {
    extern __shared__ __align__(16) unsigned char rfd_smem_[];
    __shared__ T Gs[16][17], Rl[272], rd[16];
    __shared__ double red[17];
    __shared__ int flag_s;
    const RfDenseTask<T> tk = tasks[blockIdx.x];
    const int m = tk.m, c = tk.c, maxr = tk.maxr;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nt = blockDim.x;
    T* G = (T*)rfd_smem_;                       // m x 16
    T* Y = G + (size_t)m * 16;                  // c x 17
    T* Z = Y + (size_t)c * 17;                  // maxr x 17
    T* Ut = Z + (size_t)maxr * 17;              // c x 33 (tile of U for V = B U)
    // ||Y||_F^2 (block reduction, fixed order)
    auto frob2 = [&]() -> double {
        double s = 0.0;
        for (int e = tid; e < c * 16; e += nt) { const double v = (double)Y[(e >> 4) * 17 + (e & 15)]; s += v * v; }
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) red[warp] = s;
        __syncthreads();
        if (warp == 0) {   // the warps' sums, in a fixed order, by one warp
            double t = lane < (nt >> 5) ? red[lane] : 0.0;
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            if (lane == 0) red[16] = t;
        }
        __syncthreads();
        return red[16];
    };
    // Y -= U (U^T Y) with the current rank.  Z = U^T Y: a warp per column k of U, lanes along
    // its rows (coalesced), 16 partial sums per lane folded across the warp in 16 shuffles
    // (each step halves the sums a lane keeps); lane 2q' ends with the sum of column q(lane).
    auto project = [&](int rank) {
        if (rank == 0) return;
        for (int k = warp; k < rank; k += (nt >> 5)) {
            T a[16];
#pragma unroll
            for (int q = 0; q < 16; ++q) a[q] = T(0);
            const T* uk = tk.U + (size_t)k * c;
            for (int j = lane; j < c; j += 32) {
                const T uv = uk[j];
#pragma unroll
                for (int q = 0; q < 16; ++q) a[q] = fma(uv, Y[j * 17 + q], a[q]);
            }
            const T v = rfd_fold16(a, lane);
            if ((lane & 1) == 0) Z[k * 17 + rfd_fold16_col(lane)] = v;
        }
        __syncthreads();
        for (int j = tid; j < c; j += nt) {
            T a[16];
#pragma unroll
            for (int q = 0; q < 16; ++q) a[q] = Y[j * 17 + q];
            for (int k = 0; k < rank; ++k) {
                const T uv = tk.U[j + (size_t)k * c];
#pragma unroll
                for (int q = 0; q < 16; ++q) a[q] = fma(-uv, Z[k * 17 + q], a[q]);
            }
#pragma unroll
            for (int q = 0; q < 16; ++q) Y[j * 17 + q] = a[q];
        }
        __syncthreads();
    };
    // Gram matrix Y^T Y into Gs
    auto gram = [&]() {
        if (tid < 256) {
            const int a = tid >> 4, b = tid & 15;
            T s = T(0);
            for (int j = 0; j < c; ++j) s = fma(Y[j * 17 + a], Y[j * 17 + b], s);
            Gs[a][b] = s;
        }
        __syncthreads();
    };
    // Y[:, :b] <- Y[:, :b] R^{-1} (R, 1/diag in Rl / rd), forward substitution per row
    auto rsolve = [&](int b) {
        if (tid < 16) rd[tid] = Rl[256 + tid];
        __syncthreads();
        for (int j = tid; j < c; j += nt) {
            T x[16];
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                if (q < b) {
                    T v = Y[j * 17 + q];
#pragma unroll
                    for (int k = 0; k < q; ++k) v = fma(-x[k], Rl[k * 16 + q], v);
                    x[q] = v * rd[q];
                    Y[j * 17 + q] = x[q];
                } else {
                    x[q] = T(0);
                }
            }
        }
        __syncthreads();
    };
    // warp 0 factors Gs (b x b) into Rl; returns the non-finite flag to every thread
    auto chol = [&](int b, double coef) -> bool {
        if (tid < 32) {
            const bool bad = rfp_chol(Gs, b, coef, 4.0 * max(c, 16) * tk.u, Rl);
            if (tid == 0) flag_s = bad ? 1 : 0;
        }
        __syncthreads();
        return flag_s != 0;
    };

    // row ranges of the sample product: up to three when the columns leave threads idle (the
    // partial sums of ranges 1, 2 need 2 c x 16 of the U tile's c x 33)
    const int parts = c * 3 <= nt ? 3 : (c * 2 <= nt ? 2 : 1);
    const int mpart = (m + parts - 1) / parts;
    int rank = 0;
    double y1 = 0.0;
    for (int t = 0; rank < maxr; ++t) {
        // samples of pass t and Y = B^T G
        for (int e = tid; e < m * 8; e += nt) {
            const int i = e >> 3, cp = e & 7;
            T z0, z1;
            gauss_pair<T>((uint32_t)i, (uint32_t)cp, tk.block_id, (uint32_t)t | tk.word_hi, seed, z0, z1);
            G[i * 16 + 2 * cp] = z0;
            G[i * 16 + 2 * cp + 1] = z1;
        }
        __syncthreads();
        // Y = B^T G with the rows of B split in `parts` ranges over the threads; the partial sums
        // of ranges 1, 2 go through the U tile's space (free until V = B U) and are added in order
        for (int e = tid; e < c * parts; e += nt) {
            const int j = e % c, pt = e / c;
            const int i0 = pt * mpart, i1 = min(m, i0 + mpart);
            T a[16];
#pragma unroll
            for (int q = 0; q < 16; ++q) a[q] = T(0);
            for (int i = i0; i < i1; ++i) {
                const T bv = tk.B[(size_t)i * c + j];
#pragma unroll
                for (int q = 0; q < 16; ++q) a[q] = fma(bv, G[i * 16 + q], a[q]);
            }
            T* dst = pt == 0 ? Y + (size_t)j * 17 : Ut + (size_t)(pt - 1) * c * 16 + (size_t)j * 16;
#pragma unroll
            for (int q = 0; q < 16; ++q) dst[q] = a[q];
        }
        __syncthreads();
        if (parts > 1) {
            for (int e = tid; e < c * 16; e += nt) {
                const int j = e >> 4, q = e & 15;
                T v = Y[j * 17 + q] + Ut[(size_t)j * 16 + q];
                if (parts > 2) v += Ut[(size_t)c * 16 + (size_t)j * 16 + q];
                Y[j * 17 + q] = v;
            }
            __syncthreads();
        }
        if (t == 0) y1 = sqrt(frob2());
        project(rank);
        project(rank);
        const double nrm = sqrt(frob2());
        if (!isfinite(nrm) || !isfinite(y1)) {
            if (tid == 0) atomicCAS(err, 0, 1);
            break;
        }
        if (nrm <= tk.tol * y1) break;
        const int b = min(16, maxr - rank);
        gram();
        bool bad = chol(b, 11.0 * ((double)c * b + (double)b * (b + 1)) * tk.u);
        rsolve(b);
        project(rank);
        gram();
        bad |= chol(b, 0.0);
        rsolve(b);
        gram();
        bad |= chol(b, 0.0);
        rsolve(b);
        if (bad) break;                         // non-finite pivot: drop the block's last pass
        unsigned keep = 0;
        for (int q = 0; q < b; ++q) keep |= (rd[q] != T(0) ? 1u : 0u) << q;
        const int kept = __popc(keep);
        for (int e = tid; e < c * b; e += nt) {
            const int j = e % c, q = e / c;
            if ((keep >> q) & 1u) tk.U[j + (size_t)(rank + __popc(keep & ((1u << q) - 1u))) * c] = Y[j * 17 + q];
        }
        __syncthreads();
        if (kept == 0) break;
        rank += kept;
    }
    // V = B U (m x rank, column-major), 32 columns of U staged at a time
    for (int k0 = 0; k0 < rank; k0 += 32) {
        const int kn = min(32, rank - k0);
        for (int e = tid; e < c * 32; e += nt) {
            const int j = e % c, kk = e / c;
            Ut[j * 33 + kk] = kk < kn ? tk.U[j + (size_t)(k0 + kk) * c] : T(0);
        }
        __syncthreads();
        for (int i = tid; i < m; i += nt) {
            T a[32];
#pragma unroll
            for (int kk = 0; kk < 32; ++kk) a[kk] = T(0);
            const T* bi = tk.B + (size_t)i * c;
            for (int j = 0; j < c; ++j) {
                const T bv = bi[j];
#pragma unroll
                for (int kk = 0; kk < 32; ++kk) a[kk] = fma(bv, Ut[j * 33 + kk], a[kk]);
            }
#pragma unroll
            for (int kk = 0; kk < 32; ++kk)
                if (kk < kn) tk.V[i + (size_t)(k0 + kk) * m] = a[kk];
        }
        __syncthreads();
    }
    if (tid == 0) *tk.rank = rank;
}

}  // namespace rsc
