// Tensor-core (tcgen05, sm_103a) extend-add for the BF16 and TF32 forms.
//
// One CTA (4 warps) computes a 128 x 64 tile S = A B^T of a push task, A = rows
// pr0..pr1 of L^O_k (or V_k), B = rows pc0..pc1, K = the operand's columns:
//  * each 16-wide K chunk of A and B is rounded to BF16 (or split into TF32 high and
//    low parts) and written to shared memory in the canonical K-major no-swizzle
//    layout (8 x 16-byte core matrices; K-adjacent cores 128 B apart (LBO), 8-row
//    groups 256 B apart (SBO)); a TF32 chunk is two slabs of 8 K values;
//  * one thread issues tcgen05.mma.cta_group::1.kind::f16 (M 128, N 64, K 16), or per
//    TF32 slab three kind::tf32 (K 8): A_hi B_hi + A_hi B_lo + A_lo B_hi, the
//    error-compensated split of Ootomo and Yokota (2022) that keeps the product near
//    FP32 accuracy (the A_lo B_lo term is below FP32 rounding), into an FP32
//    accumulator in tensor memory, and commits them to an mbarrier;
//  * the epilogue reads the accumulator with tcgen05.ld (warp w owns lanes 32w..32w+31
//    = rows) and scatter-adds it into the ancestor's storage like k_push.
// Every wait is bounded: on expiry the kernel records an error code, waits (bounded) for the
// MMA in flight and returns after freeing its tensor memory.
#pragma once

#include <cuda_bf16.h>
#include <cstdint>

#include "kernels.cuh"

namespace rsc {

constexpr int TC_M = 128, TC_N = 64, TC_K = 16;
constexpr unsigned long long TC_SPIN_LIMIT = 1ull << 22;
// Dynamic shared memory requested only to cap residency at 4 CTAs per SM (4 x 64 of the
// 512 tensor-memory columns), so that no CTA ever waits in tcgen05.alloc: with the static
// tiles (9.0 KB BF16, 27.0 KB split TF32) a CTA holds 50 / 57 KB of the SM's 228 KB.
constexpr int TC_PAD_SMEM = 40 * 1024;
constexpr int TC_PAD_SMEM_TF32 = 28 * 1024;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// shared-memory matrix descriptor: K-major, no swizzle, version 1 (sm_100 family)
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo & 0x3FFFF) >> 4) << 16;
    d |= (uint64_t)((sbo & 0x3FFFF) >> 4) << 32;
    d |= (uint64_t)1 << 46;           // descriptor version
    return d;                           // base offset 0, lbo mode 0, layout type 0 (no swizzle)
}

// instruction descriptors: D F32, A/B BF16 (format 1 of kind::f16) or TF32 (format 2 of
// kind::tf32), both K-major, N = 64, M = 128
constexpr uint32_t TC_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TC_N >> 3) << 17) |
                              ((uint32_t)(TC_M >> 4) << 24);
constexpr uint32_t TC_IDESC_TF32 = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TC_N >> 3) << 17) |
                                   ((uint32_t)(TC_M >> 4) << 24);

// byte offset of element (r, k) of a K-major BF16 tile with 16-element K chunks
__device__ __forceinline__ uint32_t tc_off(int r, int k) {
    return (uint32_t)(((r >> 3) * 2 + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// byte offset of the 16-byte core-matrix row holding K values 4h .. 4h + 3 of row r of a
// TF32 tile of `rows` rows: slab h / 2 (8 K values, rows x 32 bytes), core h % 2 in it
__device__ __forceinline__ uint32_t tc_off_tf32(int r, int h, int rows) {
    return (uint32_t)((h >> 1) * rows * 32 + (r >> 3) * 256 + (h & 1) * 128 + (r & 7) * 16);
}

__device__ __forceinline__ uint32_t to_tf32(float v) {   // round to nearest, ties away
    uint32_t o;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(o) : "f"(v));
    return o;
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t phase) {
    for (unsigned long long it = 0; it < TC_SPIN_LIMIT; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(bar), "r"(phase)
            : "memory");
        if (done) return true;
    }
    return false;
}

template <bool TF32>
__global__ void __launch_bounds__(128) k_push_tc(const PushTask* __restrict__ tasks, const LoOp* __restrict__ lo,
                                                 const NodeTgt* __restrict__ tgts, const int32_t* __restrict__ rows,
                                                 const long long* __restrict__ rows_ptr,
                                                 const LeafMap* __restrict__ leafmap, float* __restrict__ arena,
                                                 int* err) {
    constexpr int EB = TF32 ? 8 : 2;   // bytes per staged operand element (TF32: high and low parts)
    __shared__ __align__(1024) unsigned char As[TC_M * TC_K * EB];
    __shared__ __align__(1024) unsigned char Bs[TC_N * TC_K * EB];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_slot;
    __shared__ long long rpart[TC_M], rleaf[TC_M], cpart[TC_N], cleaf[TC_N];
    __shared__ int abort_flag;
    extern __shared__ unsigned char pad_smem[];   // occupancy limiter (tensor-memory budget)
    (void)pad_smem;

    const PushTask tk = tasks[blockIdx.x];
    const LoOp op = lo[tk.k];
    const NodeTgt tg = tgts[tk.j];
    if (tg.kind == 3 || op.K == 0) return;
    if (*(volatile int*)err) return;              // an earlier CTA already gave up
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int32_t* Rk = rows + rows_ptr[tk.k];
    const int m = tk.pr1 - tk.pr0, n = tk.pc1 - tk.pc0;
    // target maps (as in k_push)
    for (int i = tid; i < TC_M; i += blockDim.x) {
        long long rp = -1, rl = -1;
        if (i < m) {
            const long long g = Rk[tk.pr0 + i];
            const bool inC = g < tg.c0 + tg.c;
            if (tg.kind == 0) rp = inC ? g - tg.c0 : tg.c + lower_bound_i32(rows + tg.rows_off, tg.r, (int32_t)g);
            else if (inC) {
                if (tg.kind == 1) rp = g - tg.c0;
                else { const LeafMap lm = leafmap[g]; rp = g - lm.lo; rl = lm.lo; }
            }
        }
        rpart[i] = rp;
        rleaf[i] = rl;
    }
    for (int i = tid; i < TC_N; i += blockDim.x) {
        long long cp = -1, cl = -1;
        if (i < n) {
            const long long g = Rk[tk.pc0 + i];
            if (tg.kind == 0 || tg.kind == 1) cp = (g - tg.c0) * (long long)tg.ld;
            else { const LeafMap lm = leafmap[g]; cp = lm.off + (g - lm.lo) * (long long)lm.size; cl = lm.lo; }
        }
        cpart[i] = cp;
        cleaf[i] = cl;
    }
    if (warp == 0) {   // 64 TMEM columns: the 128 x 64 FP32 accumulator
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(&tmem_slot)), "r"(64) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&mbar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_flag = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;
    const float* A = (const float*)op.base + tk.pr0;
    const float* B = (const float*)op.base + tk.pc0;
    const uint32_t sa = smem_u32(As), sb = smem_u32(Bs), bar = smem_u32(&mbar);
    uint32_t phase = 0;
    int chunks = 0;
    for (int k0 = 0; k0 < op.K; k0 += TC_K) {
        // stage the chunk, zero outside the task: a thread converts 8 consecutive K values of one
        // row and stores them as one 16-byte row of a core matrix (conflict-free 16-byte stores)
        auto stage = [&](const float* src, int rows, int nr, unsigned char* dst) {
            if (TF32) {   // a thread splits 4 consecutive K values of one row: one 16-byte core row
                          // of high parts, one of low parts (the low tile follows the high one)
                for (int e = tid; e < rows * 4; e += blockDim.x) {
                    const int r = e % rows, h = e / rows;
                    uint32_t w[4], lo[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int kg = k0 + 4 * h + u;
                        const float v = (r < nr && kg < op.K) ? src[r + (size_t)kg * op.ld] : 0.f;
                        w[u] = to_tf32(v);
                        lo[u] = to_tf32(v - __uint_as_float(w[u]));
                    }
                    const uint32_t o = tc_off_tf32(r, h, rows);
                    *reinterpret_cast<uint4*>(dst + o) = make_uint4(w[0], w[1], w[2], w[3]);
                    *reinterpret_cast<uint4*>(dst + rows * TC_K * 4 + o) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
                }
                return;
            }
            for (int e = tid; e < rows * 2; e += blockDim.x) {
                const int r = e % rows, h = e / rows;     // h: K values 8h .. 8h + 7 of the chunk
                uint32_t w[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int kg0 = k0 + 8 * h + 2 * u, kg1 = kg0 + 1;
                    const float v0 = (r < nr && kg0 < op.K) ? src[r + (size_t)kg0 * op.ld] : 0.f;
                    const float v1 = (r < nr && kg1 < op.K) ? src[r + (size_t)kg1 * op.ld] : 0.f;
                    const __nv_bfloat162 b2 = __floats2bfloat162_rn(v0, v1);
                    w[u] = *reinterpret_cast<const uint32_t*>(&b2);
                }
                *reinterpret_cast<uint4*>(dst + tc_off(r, 8 * h)) = make_uint4(w[0], w[1], w[2], w[3]);
            }
        };
        stage(A, TC_M, m, As);
        stage(B, TC_N, n, Bs);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t acc = chunks > 0 ? 1u : 0u;
            if (TF32) {
                // slab sl: K values 8 sl .. 8 sl + 7 of the chunk; term t: (hi, hi), (hi, lo), (lo, hi)
#pragma unroll
                for (int q = 0; q < 6; ++q) {
                    const int sl = q / 3, t = q % 3;
                    const uint32_t a_lo = t == 2 ? TC_M * TC_K * 4 : 0, b_lo = t == 1 ? TC_N * TC_K * 4 : 0;
                    const uint64_t da = tc_desc(sa + a_lo + sl * TC_M * 32, 128, 256);
                    const uint64_t db = tc_desc(sb + b_lo + sl * TC_N * 32, 128, 256);
                    const uint32_t acc_s = q ? 1u : acc;
                    asm volatile(
                        "{\n\t.reg .pred p;\n\t"
                        "setp.ne.b32 p, %4, 0;\n\t"
                        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
                        :: "r"(tmem), "l"(da), "l"(db), "r"(TC_IDESC_TF32), "r"(acc_s) : "memory");
                }
            } else {
                const uint64_t da = tc_desc(sa, 128, 256), db = tc_desc(sb, 128, 256);
                asm volatile(
                    "{\n\t.reg .pred p;\n\t"
                    "setp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                    :: "r"(tmem), "l"(da), "l"(db), "r"(TC_IDESC), "r"(acc) : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         :: "r"(bar) : "memory");
            if (!mbar_wait(bar, phase)) {
                abort_flag = 1;
                atomicCAS(err, 0, 1);
                // keep waiting (bounded) for the MMA in flight before the tensor memory is freed;
                // a CTA may not exit holding tensor memory (a later tcgen05.alloc on this SM,
                // which cannot be bounded, would wait for it), so it is freed even if completion
                // is never observed, and the factorization reports RSC_ERR_TIMEOUT
                for (int k = 0; k < 4 && !mbar_wait(bar, phase); ++k) {}
            }
        }
        __syncthreads();
        phase ^= 1;
        ++chunks;
        if (abort_flag) break;
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!abort_flag) {
        // warp w reads rows 32w..32w+31 (its TMEM lanes), 64 FP32 columns
        uint32_t v[64];
        const uint32_t taddr = tmem + ((uint32_t)(32 * warp) << 16);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x64.b32 "
            "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
            "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,"
            "%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47,"
            "%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63}, [%64];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
              "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
              "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31]),
              "=r"(v[32]), "=r"(v[33]), "=r"(v[34]), "=r"(v[35]), "=r"(v[36]), "=r"(v[37]), "=r"(v[38]), "=r"(v[39]),
              "=r"(v[40]), "=r"(v[41]), "=r"(v[42]), "=r"(v[43]), "=r"(v[44]), "=r"(v[45]), "=r"(v[46]), "=r"(v[47]),
              "=r"(v[48]), "=r"(v[49]), "=r"(v[50]), "=r"(v[51]), "=r"(v[52]), "=r"(v[53]), "=r"(v[54]), "=r"(v[55]),
              "=r"(v[56]), "=r"(v[57]), "=r"(v[58]), "=r"(v[59]), "=r"(v[60]), "=r"(v[61]), "=r"(v[62]), "=r"(v[63])
            : "r"(taddr)
            : "memory");
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        const int i = 32 * warp + lane;
        float* dst = tg.kind == 2 ? arena : (float*)tg.base;
        if (i < m && rpart[i] >= 0) {
            const long long rp = rpart[i];
#pragma unroll
            for (int jj = 0; jj < 64; ++jj) {
                if (jj >= n) break;
                if (tk.pr0 + i < tk.pc0 + jj) continue;
                if (tg.kind == 2 && rleaf[i] != cleaf[jj]) continue;
                atomicAdd(dst + rp + cpart[jj], -__uint_as_float(v[jj]));
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(64) : "memory");
}

}  // namespace rsc
