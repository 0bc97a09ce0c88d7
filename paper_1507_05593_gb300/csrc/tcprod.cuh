// Tensor-core (tcgen05, sm_103a) thin products of the implicit sampling for the BF16 and TF32
// forms: the TN product Z = alpha A^T Y (+ beta Z) of Alg. 2 / Alg. 5 transposed and the NN
// product Y += alpha A Z (scattered rows) of Alg. 2 / Alg. 5, on FP32 storage.
//
// One CTA (4 warps) computes a 128 x NP tile of the product (NP = 16, 32 or 64 sample columns)
// as D = A_op B_op^T with both operands staged in shared memory in the canonical K-major
// no-swizzle layout (8 x 16-byte core matrices; K-adjacent cores 128 B apart, 8-row groups 256 B
// apart), 16 K values per chunk, exactly as in the tensor-core extend-add:
//  * TN: A_op[t][r] = A[r, t0 + t] (a thread reads 8 consecutive rows of one column of A: 32
//    contiguous bytes), B_op[c][r] = Y[yrow(r), c] (lanes along c: coalesced rows of Y);
//    the reduction runs over the task's rows;
//  * NN: A_op[i][l] = A[arow(i), l] (lanes along consecutive rows i of a column: coalesced),
//    B_op[c][l] = Z[l, c]; the reduction runs over the columns of A.
// BF16: operands rounded to BF16, one kind::f16 MMA (M 128, N NP, K 16) per chunk.  TF32:
// operands split into a TF32 high part and the TF32-rounded remainder, three kind::tf32 MMAs
// (K 8) per 8-wide slab, hi hi + hi lo + lo hi (Ootomo and Yokota, 2022): near FP32 accuracy.
// FP32 accumulation in tensor memory.  Two shared-memory stages: chunk i + 1 is converted and
// staged while the MMAs of chunk i run; an mbarrier per stage (tcgen05.commit) says when its
// MMAs have read it.  The epilogue reads the accumulator with tcgen05.ld (warp w owns rows
// 32 w .. 32 w + 31) and writes Z (TN; row-split partial sums added by the last CTA in a fixed
// order as in k_tn_s) or adds into Y (NN; 16-byte vector reductions where the task is atomic).
// Every wait is bounded; on expiry the kernel records an error code and, after one more
// bounded wait for the MMAs in flight, frees its tensor memory and returns.
#pragma once

#include <cuda_bf16.h>
#include <cstdint>

#include "kernels.cuh"
#include "tcgen05.cuh"

namespace rsc {

constexpr int TP_M = 128;                // rows of a product tile (columns of A for TN, rows for NN)
constexpr int TP_TMEM_COLS = 64;         // tensor-memory columns per CTA (NP <= 64 FP32 accumulators)

// bytes of one staged operand tile of `rows` rows and 16 K values
template <bool TF32> __host__ __device__ constexpr int tp_tile_bytes(int rows) { return rows * 16 * (TF32 ? 8 : 2); }
template <int NP> constexpr uint32_t tp_idesc(bool tf32) {
    return tf32 ? ((1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(NP >> 3) << 17) | ((uint32_t)(TP_M >> 4) << 24))
                : ((1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NP >> 3) << 17) | ((uint32_t)(TP_M >> 4) << 24));
}

// 8 FP32 values -> one 16-byte BF16 core row at byte offset o; or (TF32) 4 values -> a high and
// a low 16-byte core row (the low tile lo_off bytes after the high one)
__device__ __forceinline__ void tp_put_bf16(unsigned char* dst, uint32_t o, const float (&v)[8]) {
    uint32_t w[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const __nv_bfloat162 b2 = __floats2bfloat162_rn(v[2 * u], v[2 * u + 1]);
        w[u] = *reinterpret_cast<const uint32_t*>(&b2);
    }
    *reinterpret_cast<uint4*>(dst + o) = make_uint4(w[0], w[1], w[2], w[3]);
}
__device__ __forceinline__ void tp_put_tf32(unsigned char* dst, uint32_t o, uint32_t lo_off, const float* v) {
    uint32_t hi[4], lo[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        hi[u] = to_tf32(v[u]);
        lo[u] = to_tf32(v[u] - __uint_as_float(hi[u]));
    }
    *reinterpret_cast<uint4*>(dst + o) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
    *reinterpret_cast<uint4*>(dst + lo_off + o) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
}
// issue the MMAs of one staged chunk (thread 0)
template <bool TF32, int NP>
__device__ __forceinline__ void tp_mma(uint32_t tmem, uint32_t sa, uint32_t sb, bool accumulate) {
    if (TF32) {
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            const int sl = q / 3, t = q % 3;   // slab, term: (hi, hi), (hi, lo), (lo, hi)
            const uint32_t a_lo = t == 2 ? TP_M * 16 * 4 : 0, b_lo = t == 1 ? NP * 16 * 4 : 0;
            const uint64_t da = tc_desc(sa + a_lo + sl * TP_M * 32, 128, 256);
            const uint64_t db = tc_desc(sb + b_lo + sl * NP * 32, 128, 256);
            const uint32_t acc = (q > 0 || accumulate) ? 1u : 0u;
            asm volatile(
                "{\n\t.reg .pred p;\n\t"
                "setp.ne.b32 p, %4, 0;\n\t"
                "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
                :: "r"(tmem), "l"(da), "l"(db), "r"(tp_idesc<NP>(true)), "r"(acc) : "memory");
        }
    } else {
        const uint64_t da = tc_desc(sa, 128, 256), db = tc_desc(sb, 128, 256);
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
            :: "r"(tmem), "l"(da), "l"(db), "r"(tp_idesc<NP>(false)), "r"(accumulate ? 1u : 0u) : "memory");
    }
}
// 16 FP32 accumulator columns c0 .. c0 + 15 of this thread's row
__device__ __forceinline__ void tp_ld16(uint32_t taddr, float (&o)[16]) {
    uint32_t v[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int q = 0; q < 16; ++q) o[q] = __uint_as_float(v[q]);
}

// ------------------------------------------------------------------ pipeline
// Raw FP32 chunks of KC reduction values stream through a ring of TP_STAGES shared-memory
// stages by cp.async (two chunks ahead of the one being converted); each chunk is then
// converted shared-to-shared into the K-major BF16 / TF32 operand layout of one of two operand
// buffers, whose MMAs are committed to that buffer's mbarrier, so the loads of chunks i + 1 and
// i + 2, the conversion of chunk i and the MMAs of chunk i - 1 overlap.
constexpr int TP_STAGES = 3;
template <bool TF32> __host__ __device__ constexpr int tp_kc() { return TF32 ? 16 : 32; }
// operand buffer: KC / 16 sub-tiles of 16 K values, A (128 rows) then B (NP rows)
template <bool TF32> __host__ __device__ constexpr int tp_op_bytes(int np) {
    return (tp_kc<TF32>() / 16) * (tp_tile_bytes<TF32>(TP_M) + tp_tile_bytes<TF32>(np));
}
// raw stage: A as [128][KC + 4] floats (TN) or [KC][128 + 4] (NN), B as [KC][NP + 4] floats
template <bool TF32> __host__ __device__ constexpr int tp_raw_bytes(int np) {
    return 4 * ((TP_M + 4) * (tp_kc<TF32>() + 4) > (tp_kc<TF32>() * (TP_M + 4))
                    ? (TP_M + 4) * (tp_kc<TF32>() + 4) + tp_kc<TF32>() * (np + 4)
                    : tp_kc<TF32>() * (TP_M + 4) + tp_kc<TF32>() * (np + 4));
}
template <bool TF32> __host__ __device__ constexpr int tp_smem2(int np) {
    return 2 * ((tp_op_bytes<TF32>(np) + 1023) / 1024 * 1024) + TP_STAGES * ((tp_raw_bytes<TF32>(np) + 127) / 128 * 128);
}
template <bool TF32> __host__ __device__ constexpr int tp_smem_bytes(int np) {
    return tp_smem2<TF32>(np) > 28 * 1024 ? tp_smem2<TF32>(np) : 28 * 1024;
}

// issue the MMAs of one converted chunk (thread 0): KC / 16 steps of 16 K values
template <bool TF32, int NP>
__device__ __forceinline__ void tp_mma_chunk(uint32_t tmem, uint32_t op, bool accumulate) {
    constexpr int SA = tp_tile_bytes<TF32>(TP_M), SBB = tp_tile_bytes<TF32>(NP);
#pragma unroll
    for (int st = 0; st < tp_kc<TF32>() / 16; ++st) {
        const uint32_t a = op + st * (SA + SBB), b = a + SA;
        tp_mma<TF32, NP>(tmem, a, b, accumulate || st > 0);
    }
}

// convert element (row, k) of a raw tile given by `val` into the operand sub-tiles at dst
// (rows x KC), a thread per (row, 8-value group) with row fastest
template <bool TF32, class F>
__device__ __forceinline__ void tp_convert(unsigned char* dst, int rows, int stride_sub, F&& val) {
    constexpr int KC = tp_kc<TF32>();
    for (int e = threadIdx.x; e < rows * (KC / 8); e += blockDim.x) {
        const int r = e % rows, g = e / rows;          // K values 8 g .. 8 g + 7
        const int st = g >> 1, h = g & 1;              // 16-value sub-tile, half in it
        float v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = val(r, 8 * g + u);
        unsigned char* sub = dst + st * stride_sub;
        if (TF32) {
            const uint32_t lo_off = (uint32_t)rows * 16 * 4;
            tp_put_tf32(sub, tc_off_tf32(r, 2 * h, rows), lo_off, v);
            tp_put_tf32(sub, tc_off_tf32(r, 2 * h + 1, rows), lo_off, v + 4);
        } else {
            tp_put_bf16(sub, tc_off(r, 8 * h), v);
        }
    }
}

__device__ __forceinline__ void tp_cp_wait(int pending) {
    if (pending >= 2) cp_async_wait<2>();
    else if (pending == 1) cp_async_wait<1>();
    else cp_async_wait<0>();
}

// The chunk loop shared by both products.  load(ci, raw) issues the cp.async copies of chunk ci
// into a raw stage (and zero-fills its rows past the end); conv(raw, op) converts a landed
// chunk.  Returns false when a wait ran out (the error word is set).
template <bool TF32, int NP, class LOAD, class CONV>
__device__ bool tp_pipeline(int nchunk, unsigned char* smem, uint32_t tmem, uint64_t* mbar, int* abort_s, int* err,
                            LOAD&& load, CONV&& conv) {
    const int tid = threadIdx.x;
    constexpr int OPB = (tp_op_bytes<TF32>(NP) + 1023) / 1024 * 1024;
    constexpr int RAWB = (tp_raw_bytes<TF32>(NP) + 127) / 128 * 128;
    unsigned char* raw0 = smem + 2 * OPB;
    uint32_t phase = 0u, outstanding = 0u;   // bit b: parity to wait for / MMAs in flight on operand buffer b
    auto give_up = [&]() {                   // more bounded waits for the MMAs in flight, then report
        if (tid == 0)
            for (int b = 0; b < 2; ++b)
                if ((outstanding >> b) & 1u)
                    for (int k = 0; k < 4 && !mbar_wait(smem_u32(&mbar[b]), (phase >> b) & 1u); ++k) {}
        __syncthreads();
        return false;
    };
    for (int ci = 0; ci < min(2, nchunk); ++ci) { load(ci, raw0 + ci * RAWB); cp_async_commit(); }
    for (int ci = 0; ci < nchunk; ++ci) {
        if (ci + 2 < nchunk) { load(ci + 2, raw0 + ((ci + 2) % TP_STAGES) * RAWB); cp_async_commit(); }
        tp_cp_wait(min(2, nchunk - 1 - ci));
        const int b = ci & 1;
        if ((outstanding >> b) & 1u) {       // the MMAs of chunk ci - 2 read operand buffer b
            if (tid == 0 && !mbar_wait(smem_u32(&mbar[b]), (phase >> b) & 1u)) {
                *abort_s = 1;
                atomicCAS(err, 0, 1);
            }
        }
        __syncthreads();
        if (*abort_s) return give_up();
        if ((outstanding >> b) & 1u) { phase ^= 1u << b; outstanding &= ~(1u << b); }
        conv(raw0 + (ci % TP_STAGES) * RAWB, smem + b * OPB);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            tp_mma_chunk<TF32, NP>(tmem, smem_u32(smem + b * OPB), ci > 0);
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         :: "r"(smem_u32(&mbar[b])) : "memory");
        }
        outstanding |= 1u << b;
    }
    for (int b = 0; b < 2; ++b) {
        if (!((outstanding >> b) & 1u)) continue;
        if (tid == 0) {
            if (mbar_wait(smem_u32(&mbar[b]), (phase >> b) & 1u)) outstanding &= ~(1u << b);
            else { *abort_s = 1; atomicCAS(err, 0, 1); }
        }
    }
    __syncthreads();
    if (*abort_s) return give_up();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    return true;
}

// tensor-memory allocation (warp 0) and mbarrier set-up; all threads synced on return
__device__ __forceinline__ uint32_t tp_begin(uint32_t* tmem_slot, uint64_t* mbar, int* abort_s) {
    if ((threadIdx.x >> 5) == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(tmem_slot)), "r"(TP_TMEM_COLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&mbar[0])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&mbar[1])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *abort_s = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    return *tmem_slot;
}
// free the tensor memory (every MMA has completed, or its waits have run out: see tp_pipeline)
__device__ __forceinline__ void tp_end(uint32_t tmem) {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if ((threadIdx.x >> 5) == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(TP_TMEM_COLS) : "memory");
}

// ------------------------------------------------------------------ TN: Z = alpha A^T Y + beta Z
// Grid (tasks, 64-column chunks of Y, row splits); a task covers columns t0 .. t0 + 127 of A.
// Raw stage: Ar[t][r] (t < 128, r < KC; a warp copies KC consecutive rows of one column),
// Yr[r][c] (the gathered rows of Y).
template <bool TF32, int NP>
__global__ void __launch_bounds__(128) k_tn_tc(const TnTask* __restrict__ tasks, int* err) {
    extern __shared__ __align__(1024) unsigned char tp_smem[];
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_s, last;
    constexpr int KC = tp_kc<TF32>(), AST = KC + 4, YST = NP + 4;
    constexpr int SUB = tp_tile_bytes<TF32>(TP_M) + tp_tile_bytes<TF32>(NP);   // one 16-K sub-tile (A + B)
    const TnTask tk = tasks[blockIdx.x];
    const int cb = blockIdx.y * 64;
    const int nc = min(64, tk.N - cb);
    if (nc <= 0 || (int)blockIdx.z >= tk.nsplit) return;
    if (*(volatile int*)err) return;              // an earlier CTA already gave up
    const int tid = threadIdx.x;
    const int rb = (int)blockIdx.z * tk.rps;
    const int re = tk.nsplit > 1 ? min(tk.nrow, rb + tk.rps) : tk.nrow;
    const int kc = min(TP_M, tk.K - tk.t0);
    const float* A = (const float*)tk.A + (size_t)tk.t0 * tk.lda;
    const float* Y = (const float*)tk.Y + cb;
    const bool yvec = (nc % 4) == 0 && (tk.ldy % 4) == 0 && (((uintptr_t)Y) & 15) == 0;
    const uint32_t tmem = tp_begin(&tmem_slot, mbar, &abort_s);
    const int nchunk = re > rb ? (re - rb + KC - 1) / KC : 0;
    auto load = [&](int ci, unsigned char* raw) {
        float* Ar = (float*)raw;
        float* Yr = Ar + TP_M * AST;
        const int r0 = rb + ci * KC, rc = min(KC, re - r0);
        // A: 16-byte copies down a column where the rows are contiguous and aligned
        const bool avec = !tk.amap && rc == KC && (tk.lda % 4) == 0 && (((uintptr_t)(A + tk.aoff + r0)) & 15) == 0;
        if (avec) {
            for (int e = tid; e < TP_M * (KC / 4); e += blockDim.x) {
                const int q = e % (KC / 4), t = e / (KC / 4);
                if (t < kc) cp_async16(Ar + t * AST + 4 * q, A + (size_t)t * tk.lda + tk.aoff + r0 + 4 * q);
            }
        } else {
            for (int e = tid; e < TP_M * KC; e += blockDim.x) {
                const int r = e % KC, t = e / KC;
                if (t < kc && r < rc) {
                    const int i = r0 + r;
                    const int ar = (tk.amap ? tk.amap[i] : i) + tk.aoff;
                    cp_async4(Ar + t * AST + r, A + (size_t)t * tk.lda + ar);
                } else if (r >= rc) {
                    Ar[t * AST + r] = 0.f;
                }
            }
        }
        if (yvec) {
            const int per = nc / 4;
            for (int e = tid; e < KC * per; e += blockDim.x) {
                const int r = e / per, q = e % per;
                if (r < rc) {
                    const int i = r0 + r;
                    const int yr = (tk.ymap ? tk.ymap[i] : i) + tk.yoff;
                    cp_async16(Yr + r * YST + 4 * q, Y + (size_t)yr * tk.ldy + 4 * q);
                }
            }
        } else {
            for (int e = tid; e < KC * nc; e += blockDim.x) {
                const int r = e / nc, c = e % nc;
                if (r < rc) {
                    const int i = r0 + r;
                    const int yr = (tk.ymap ? tk.ymap[i] : i) + tk.yoff;
                    cp_async4(Yr + r * YST + c, Y + (size_t)yr * tk.ldy + c);
                }
            }
        }
        if (rc < KC)
            for (int e = tid; e < (KC - rc) * YST; e += blockDim.x) Yr[rc * YST + e] = 0.f;
    };
    auto conv = [&](unsigned char* raw, unsigned char* op) {
        const float* Ar = (const float*)raw;
        const float* Yr = Ar + TP_M * AST;
        tp_convert<TF32>(op, TP_M, SUB, [&](int t, int k) -> float { return Ar[t * AST + k]; });
        tp_convert<TF32>(op + tp_tile_bytes<TF32>(TP_M), NP, SUB, [&](int c, int k) -> float { return Yr[k * YST + c]; });
    };
    bool ok = true;
    if (nchunk > 0) ok = tp_pipeline<TF32, NP>(nchunk, tp_smem, tmem, mbar, &abort_s, err, load, conv);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int t = 32 * warp + lane;              // this thread's row of the tile (column of A)
    if (ok) {
        float acc[NP];
        if (nchunk > 0) {
#pragma unroll
            for (int q0 = 0; q0 < NP; q0 += 16) {
                float o[16];
                tp_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)q0, o);
#pragma unroll
                for (int q = 0; q < 16; ++q) acc[q0 + q] = o[q];
            }
        } else {
#pragma unroll
            for (int q = 0; q < NP; ++q) acc[q] = 0.f;
        }
        if (tk.nsplit == 1) {
            if (t < kc) {
                float* z = (float*)tk.Z + (size_t)(tk.t0 + t) * tk.ldz + cb;
#pragma unroll
                for (int q = 0; q < NP; ++q)
                    if (q < nc) z[q] = tk.beta != 0.0 ? (float)tk.beta * z[q] + (float)tk.alpha * acc[q]
                                                      : (float)tk.alpha * acc[q];
            }
        } else {
            float* part = (float*)tk.part;
#pragma unroll
            for (int q = 0; q < NP; ++q)
                if (q < nc) part[((size_t)blockIdx.z * TP_M + t) * tk.N + cb + q] = acc[q];
            __threadfence();
            __syncthreads();
            if (threadIdx.x == 0) last = atomicAdd(tk.cnt + blockIdx.y, 1u) == (unsigned)(tk.nsplit - 1);
            __syncthreads();
            if (last) {
                __threadfence();
                for (int e = threadIdx.x; e < kc * nc; e += blockDim.x) {
                    const int tt = e / nc, c = e % nc;
                    float s = 0.f;
                    for (int zz = 0; zz < tk.nsplit; ++zz) s += __ldcg((float*)tk.part + ((size_t)zz * TP_M + tt) * tk.N + cb + c);
                    float* z = (float*)tk.Z + (size_t)(tk.t0 + tt) * tk.ldz + cb + c;
                    *z = tk.beta != 0.0 ? (float)tk.beta * *z + (float)tk.alpha * s : (float)tk.alpha * s;
                }
                if (threadIdx.x == 0) tk.cnt[blockIdx.y] = 0u;
            }
        }
    }
    tp_end(tmem);
}

// ------------------------------------------------------------------ NN: Y[yrow_i, :] += alpha A[arow_i, :] Z
// Grid (tasks, 64-column chunks of Z); a task covers rows row0 .. row0 + 127.  Raw stage:
// Ar[l][i] (a warp copies consecutive rows of one column of A), Zr[l][c].
template <bool TF32, int NP>
__global__ void __launch_bounds__(128) k_nn_tc(const NnTask* __restrict__ tasks, int* err) {
    extern __shared__ __align__(1024) unsigned char tp_smem[];
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_s;
    constexpr int KC = tp_kc<TF32>(), AST = TP_M + 4, ZST = NP + 4;
    constexpr int SUB = tp_tile_bytes<TF32>(TP_M) + tp_tile_bytes<TF32>(NP);
    const NnTask tk = tasks[blockIdx.x];
    const int cb = blockIdx.y * 64;
    const int nc = min(64, tk.N - cb);
    if (nc <= 0 || tk.K <= 0) return;
    if (*(volatile int*)err) return;
    const int tid = threadIdx.x;
    const int mr = min(TP_M, tk.nrow - tk.row0);
    const float* A = (const float*)tk.A;
    const float* Z = (const float*)tk.Z + cb;
    const bool zvec = (nc % 4) == 0 && (tk.ldz % 4) == 0 && (((uintptr_t)Z) & 15) == 0;
    const int arow0 = (tk.amap ? 0 : tk.row0 + tk.aoff);
    const bool avec = !tk.amap && mr == TP_M && (tk.lda % 4) == 0 && (((uintptr_t)(A + arow0)) & 15) == 0;
    const uint32_t tmem = tp_begin(&tmem_slot, mbar, &abort_s);
    const int nchunk = (tk.K + KC - 1) / KC;
    auto load = [&](int ci, unsigned char* raw) {
        float* Ar = (float*)raw;
        float* Zr = Ar + KC * AST;
        const int l0 = ci * KC, lc = min(KC, tk.K - l0);
        if (avec) {
            for (int e = tid; e < KC * (TP_M / 4); e += blockDim.x) {
                const int q = e % (TP_M / 4), l = e / (TP_M / 4);
                if (l < lc) cp_async16(Ar + l * AST + 4 * q, A + arow0 + (size_t)(l0 + l) * tk.lda + 4 * q);
                else *reinterpret_cast<float4*>(Ar + l * AST + 4 * q) = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        } else {
            for (int e = tid; e < KC * TP_M; e += blockDim.x) {
                const int i = e % TP_M, l = e / TP_M;
                if (l < lc && i < mr) {
                    const int ii = tk.row0 + i;
                    const int ar = (tk.amap ? tk.amap[ii] : ii) + tk.aoff;
                    cp_async4(Ar + l * AST + i, A + ar + (size_t)(l0 + l) * tk.lda);
                } else if (l >= lc) {
                    Ar[l * AST + i] = 0.f;
                }
            }
        }
        if (zvec) {
            const int per = nc / 4;
            for (int e = tid; e < KC * per; e += blockDim.x) {
                const int l = e / per, q = e % per;
                if (l < lc) cp_async16(Zr + l * ZST + 4 * q, Z + (size_t)(l0 + l) * tk.ldz + 4 * q);
            }
        } else {
            for (int e = tid; e < KC * nc; e += blockDim.x) {
                const int l = e / nc, c = e % nc;
                if (l < lc) cp_async4(Zr + l * ZST + c, Z + (size_t)(l0 + l) * tk.ldz + c);
            }
        }
        if (lc < KC)
            for (int e = tid; e < (KC - lc) * ZST; e += blockDim.x) Zr[lc * ZST + e] = 0.f;
    };
    auto conv = [&](unsigned char* raw, unsigned char* op) {
        const float* Ar = (const float*)raw;
        const float* Zr = Ar + KC * AST;
        tp_convert<TF32>(op, TP_M, SUB, [&](int i, int k) -> float { return Ar[k * AST + i]; });
        tp_convert<TF32>(op + tp_tile_bytes<TF32>(TP_M), NP, SUB, [&](int c, int k) -> float { return Zr[k * ZST + c]; });
    };
    const bool ok = tp_pipeline<TF32, NP>(nchunk, tp_smem, tmem, mbar, &abort_s, err, load, conv);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i = 32 * warp + lane;
    if (ok) {
        float acc[NP];
#pragma unroll
        for (int q0 = 0; q0 < NP; q0 += 16) {   // every lane of the warp takes part in tcgen05.ld
            float o[16];
            tp_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)q0, o);
#pragma unroll
            for (int q = 0; q < 16; ++q) acc[q0 + q] = o[q];
        }
        if (i < mr) {
            const int ii = tk.row0 + i;
            const int yr = (tk.ymap ? tk.ymap[ii] : ii) + tk.yoff;
            float* y = (float*)tk.Y + (size_t)yr * tk.ldy + cb;
            const float alpha = (float)tk.alpha;
            const bool vec = (nc % 4) == 0 && (((uintptr_t)y) & 15) == 0;
#pragma unroll
            for (int q = 0; q < NP; q += 4) {
                if (q >= nc) break;
                if (tk.atomic && vec) {
                    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};"
                                 :: "l"(y + q), "f"(alpha * acc[q]), "f"(alpha * acc[q + 1]), "f"(alpha * acc[q + 2]),
                                    "f"(alpha * acc[q + 3]) : "memory");
                } else {
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        if (q + u >= nc) break;
                        if (tk.atomic) atomicAdd(y + q + u, alpha * acc[q + u]);
                        else y[q + u] += alpha * acc[q + u];
                    }
                }
            }
        }
    }
    tp_end(tmem);
}

}  // namespace rsc
