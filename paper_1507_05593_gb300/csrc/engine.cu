// GPU engine: plan building, the level-scheduled factorization (Algorithms 1-6)
// and the PCG solve with the two triangular solves as preconditioner.
//
// Factorization schedule (one pass per level of the supernodal elimination tree):
//   1. uncompressed supernodes (and compressed ones with a dense diagonal) of the
//      level factor their dense panels [L^D_j; L^O_j] by a blocked tall-panel
//      Cholesky (diagonal-tile POTRF, TRSM of the rows below, trailing update),
//      batched over the level;
//   2. compressed supernodes of the level build their hierarchical diagonal
//      blocks (Alg. 6 for leaves, Alg. 5 + adaptive range finder for the others)
//      and their off-diagonal low-rank blocks (Alg. 2, 3), one supernode at a time;
//   3. every supernode of the level pushes its Schur update
//      L^O_k L^O_k^T (or V_k V_k^T) into its ancestors' dense storage (the
//      extend-add of Eqs. "schurDiag"/"schurOffDiag", Alg. 1) with atomic adds.
// The uncompressed target of supernode j therefore holds U^D_j and U^O_j of Alg. 1
// when step 1 reaches it; compressed targets only receive the entries of their
// dense diagonal storage, the rest is applied implicitly by Alg. 2 / Alg. 5.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <cstdio>
#include <map>
#include <tuple>
#include <atomic>
#include <mutex>
#include <functional>
#include <numeric>

#include <chrono>

#include "engine.h"
#include "kernels.cuh"
#include "tcgen05.cuh"
#include "rfpass.cuh"
#include "tcprod.cuh"

namespace rsc {

#define CK(x)                                                                                    \
    do {                                                                                         \
        cudaError_t e_ = (x);                                                                    \
        if (e_ != cudaSuccess)                                                                   \
            throw Error(e_ == cudaErrorMemoryAllocation ? RSC_ERR_OOM : RSC_ERR_CUDA,             \
                        std::string(#x) + ": " + cudaGetErrorString(e_));                        \
    } while (0)

#define LAUNCH_CHECK() CK(cudaGetLastError())

static inline int cdiv(long long a, long long b) { return (int)((a + b - 1) / b); }

// ------------------------------------------------------------------ device memory
class DeviceMem {
public:
    ~DeviceMem() { release(); }
    void* alloc(size_t bytes) {
        if (bytes == 0) bytes = 16;
        bytes = (bytes + 255) / 256 * 256;
        // a block kept by recycle() of the same size class (bytes .. 2 bytes), smallest first
        int bi = -1;
        for (int i = 0; i < (int)free_.size(); ++i)
            if (free_[i].second >= bytes && free_[i].second <= 2 * bytes &&
                (bi < 0 || free_[i].second < free_[bi].second))
                bi = i;
        if (bi >= 0) {
            const auto b = free_[bi];
            free_.erase(free_.begin() + bi);
            ptrs_.push_back(b.first);
            sizes_.push_back(b.second);
            total_ += b.second;
            return b.first;
        }
        void* p = nullptr;
        CK(cudaMalloc(&p, bytes));
        ptrs_.push_back(p);
        sizes_.push_back(bytes);
        total_ += bytes;
        return p;
    }
    // keep every block for the next allocations of the same sizes (a launch list rebuilt
    // after each factorization), instead of freeing and allocating them again
    void recycle() {
        for (size_t i = 0; i < ptrs_.size(); ++i) free_.emplace_back(ptrs_[i], sizes_[i]);
        ptrs_.clear();
        sizes_.clear();
        total_ = 0;
    }
    void trim() {   // free the kept blocks that no allocation took
        for (auto& b : free_) cudaFree(b.first);
        free_.clear();
    }
    template <class X> X* upload(const std::vector<X>& v, cudaStream_t s) {
        X* p = (X*)alloc(sizeof(X) * std::max<size_t>(v.size(), 1));
        if (!v.empty()) CK(cudaMemcpyAsync(p, v.data(), sizeof(X) * v.size(), cudaMemcpyHostToDevice, s));
        return p;
    }
    void release() {
        for (void* p : ptrs_) cudaFree(p);
        ptrs_.clear();
        sizes_.clear();
        total_ = 0;
        trim();
    }
    size_t total() const { return total_; }

private:
    std::vector<void*> ptrs_;
    std::vector<size_t> sizes_;
    std::vector<std::pair<void*, size_t>> free_;
    size_t total_ = 0;
};

// growable device scratch
struct Scratch {
    void* p = nullptr;
    size_t bytes = 0;
    ~Scratch() { if (p) cudaFree(p); }
    void* get(size_t b) {
        if (b > bytes) {
            if (p) CK(cudaFree(p));
            p = nullptr;
            size_t nb = std::max(b, bytes * 3 / 2);
            CK(cudaMalloc(&p, nb));
            bytes = nb;
        }
        return p;
    }
};

// ------------------------------------------------------------------ kernel profiler
// CUDA event pairs around launches of the enabled kernel classes; per class the
// launch count, device time and the algorithmic flops and bytes of the launches.
struct Profiler {
    bool on = false;
    std::string only;      // empty: every class; else a comma-separated list of class names
    struct Pend { std::string name; cudaEvent_t a, b; double flops, bytes; };
    std::string tag;       // appended to the class names of later launches (e.g. the level)
    struct Acc { long long n = 0; double ms = 0, flops = 0, bytes = 0; };
    std::vector<cudaEvent_t> pool;
    std::vector<Pend> pend;
    std::map<std::string, Acc> acc;
    ~Profiler() {
        for (auto& p : pend) { pool.push_back(p.a); pool.push_back(p.b); }
        if (lastb) pool.push_back(lastb);
        for (cudaEvent_t e : pool) cudaEventDestroy(e);
    }
    bool enabled(const char* name) const {
        if (!on) return false;
        if (only.empty()) return true;
        std::string key = std::string(",") + only + ",";
        return key.find(std::string(",") + name + ",") != std::string::npos;
    }
    cudaEvent_t ev() {
        if (pool.empty()) { cudaEvent_t e; CK(cudaEventCreate(&e)); return e; }
        cudaEvent_t e = pool.back(); pool.pop_back(); return e;
    }
    cudaEvent_t lastb = nullptr;   // end of the previous recorded launch (idle-gap accounting)
    void mark() {                  // forget the previous launch: the next gap is not counted
        if (lastb) pool.push_back(lastb);
        lastb = nullptr;
    }
    void flush() {
        if (pend.empty()) return;
        CK(cudaEventSynchronize(pend.back().b));
        for (auto& p : pend) {
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, p.a, p.b));
            Acc& a = acc[p.name];
            a.n++; a.ms += ms; a.flops += p.flops; a.bytes += p.bytes;
            if (lastb) {   // device idle (or other work) between the previous launch and this one
                float g = 0.f;
                CK(cudaEventElapsedTime(&g, lastb, p.a));
                Acc& ga = acc["gap>" + p.name];
                ga.n++; ga.ms += g;
                pool.push_back(lastb);
            }
            pool.push_back(p.a);
            lastb = p.b;
        }
        pend.clear();
    }
    // host wall time of a phase (stream drained at both ends), kept beside the kernel classes
    void wall(const std::string& name, double ms) {
        if (!on) return;
        Acc& a = acc[name];
        a.n++; a.ms += ms;
    }
    std::string json() {
        flush();
        std::string out = "{";
        bool first = true;
        char buf[256];
        for (auto& kv : acc) {
            std::snprintf(buf, sizeof(buf), "%s\"%s\": {\"launches\": %lld, \"ms\": %.6f, \"flops\": %.6e, \"bytes\": %.6e}",
                          first ? "" : ", ", kv.first.c_str(), kv.second.n, kv.second.ms, kv.second.flops, kv.second.bytes);
            out += buf;
            first = false;
        }
        return out + "}";
    }
};

#define PROF(P, NAME, STREAM, FLOPS, BYTES, ...)                                   \
    do {                                                                       \
        if ((P).enabled(NAME)) {                                               \
            cudaEvent_t a_ = (P).ev(), b_ = (P).ev();                          \
            CK(cudaEventRecord(a_, STREAM));                                   \
            __VA_ARGS__;                                                       \
            CK(cudaEventRecord(b_, STREAM));                                   \
            (P).pend.push_back({std::string(NAME) + (P).tag, a_, b_, (double)(FLOPS), (double)(BYTES)}); \
        } else {                                                               \
            __VA_ARGS__;                                                       \
        }                                                                      \
    } while (0)

// ------------------------------------------------------------------ kernel-variant tuner
// Autotuning of the thin products' kernel (SIMT or tensor cores, which differ in tile shape:
// 64 or 128 columns of A per CTA, 16 or 64 sample columns per CTA) per (class, padded sample
// width, log2 of the launch's flops).  During a handle's first factorization in a form that has
// both kernels, the launches of each key alternate between the variants and are timed with CUDA
// events; after that factorization every key takes the variant with the smaller time per flop
// (keys seen with one variant only, or never, take the default).  Every launch runs exactly one
// variant, so the tuned factorization computes the same factor as any other.
struct Tuner {
    bool tuning = false;
    struct Stat { double sec[2] = {0, 0}, flops[2] = {0, 0}; int n[2] = {0, 0}; int choice = -1; };
    std::map<std::string, Stat> tab;
    struct Pend { std::string key; int var; double flops; cudaEvent_t a, b; };
    std::vector<Pend> pend;
    std::vector<cudaEvent_t> pool;
    ~Tuner() {
        for (auto& p : pend) { pool.push_back(p.a); pool.push_back(p.b); }
        for (cudaEvent_t e : pool) cudaEventDestroy(e);
    }
    static std::string key(const char* cls, int np, double flops) {
        const int b = flops > 1.0 ? (int)std::floor(std::log2(flops)) : 0;
        return std::string(cls) + "/n" + std::to_string(np) + "/2^" + std::to_string(b);
    }
    int pick(const std::string& k, int dflt) {
        if (tuning) {
            const Stat& st = tab[k];
            return st.n[1] < st.n[0] ? 1 : 0;
        }
        auto it = tab.find(k);
        return (it != tab.end() && it->second.choice >= 0) ? it->second.choice : dflt;
    }
    cudaEvent_t ev() {
        if (pool.empty()) { cudaEvent_t e; CK(cudaEventCreate(&e)); return e; }
        cudaEvent_t e = pool.back(); pool.pop_back(); return e;
    }
    struct Timed {   // events around one launch while tuning (empty key: not a tuned launch)
        Tuner& t; bool on; cudaStream_t s; Pend p{};
        Timed(Tuner& t_, const std::string& k, int var, double fl, cudaStream_t s_)
            : t(t_), on(t_.tuning && !k.empty()), s(s_) {
            if (!on) return;
            p.key = k; p.var = var; p.flops = fl; p.a = t.ev(); p.b = t.ev();
            t.tab[k].n[var]++;
            CK(cudaEventRecord(p.a, s));
        }
        ~Timed() {
            if (!on) return;
            if (cudaEventRecord(p.b, s) == cudaSuccess) t.pend.push_back(p);
        }
    };
    // after the tuning factorization (stream idle): collect the times, choose per key
    void finish() {
        for (auto& p : pend) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
                Stat& st = tab[p.key];
                st.sec[p.var] += ms * 1e-3;
                st.flops[p.var] += p.flops;
            }
            pool.push_back(p.a);
            pool.push_back(p.b);
        }
        pend.clear();
        for (auto& kv : tab) {
            Stat& st = kv.second;
            if (st.flops[0] > 0 && st.flops[1] > 0)
                st.choice = st.sec[1] / st.flops[1] < st.sec[0] / st.flops[0] ? 1 : 0;
        }
        tuning = false;
    }
    // a factorization that failed: drop its timings (tuning resumes with the next one)
    void abandon() {
        for (auto& p : pend) { pool.push_back(p.a); pool.push_back(p.b); }
        pend.clear();
        for (auto& kv : tab) kv.second.n[0] = kv.second.n[1] = 0;
        tuning = false;
    }
    std::string json() const {
        std::string out = "{";
        char buf[320];
        bool first = true;
        for (auto& kv : tab) {
            const Stat& st = kv.second;
            std::snprintf(buf, sizeof(buf),
                          "%s\"%s\": {\"choice\": %d, \"simt_ns_per_mflop\": %.3f, \"tensor_ns_per_mflop\": %.3f, "
                          "\"launches\": [%d, %d]}",
                          first ? "" : ", ", kv.first.c_str(), st.choice,
                          st.flops[0] > 0 ? st.sec[0] / st.flops[0] * 1e15 : -1.0,
                          st.flops[1] > 0 ? st.sec[1] / st.flops[1] * 1e15 : -1.0, st.n[0], st.n[1]);
            out += buf;
            first = false;
        }
        return out + "}";
    }
};

// ------------------------------------------------------------------ engine base
struct EngineImpl {
    Tuner tuner;
    bool tuned_once = false;
    // polls of a grid-barrier wait of the cooperative range-finder kernel before it gives up
    unsigned long long rf_spin_limit = RFP_SPIN_LIMIT;
    // values given on the device (rsc_refactor_values_device): the caller's order, nnz entries;
    // while vals_dev is set they, not the host copy, feed the factorization and the SpMV
    DeviceMem umem;
    double* d_uval = nullptr;
    long long n_uval = 0;
    bool vals_dev = false;
    void set_values_device(const double* d_val, long long nnz, cudaStream_t s);
    Profiler prof;
    virtual ~EngineImpl() = default;
    virtual rsc_status factor(const double* val, double tol, const FixedRank* fr) = 0;
    virtual bool factored() const = 0;
    virtual void apply(const double* d_r, double* d_z, cudaStream_t s) = 0;
    virtual void prepare_multi(int) {}
    virtual void apply_multi(const double* d_r, double* d_z, int nrhs, cudaStream_t s) {
        for (int c = 0; c < nrhs; ++c) apply(d_r + (size_t)c * n_of(), d_z + (size_t)c * n_of(), s);
    }
    virtual long long n_of() const = 0;
    virtual void node_info(int j, int32_t* info) const = 0;
    virtual rsc_status node_blocks(int j, double* LD, double* LO) = 0;
    virtual void stats(rsc_stats_t* out) const = 0;
    virtual long long generation() const = 0;
    long long uid = 0;    // unique per engine (never reused, unlike its address)
    int device = 0;       // the CUDA device the engine's memory and stream belong to
    virtual rsc_status apply_noalloc(const double* d_r, double* d_z, cudaStream_t s, char* base, size_t cap,
                                     bool load) = 0;
    virtual bool noalloc_ready() const = 0;
    // PCG state shared by every precision
    void ensure_matrix(const std::vector<int64_t>& rp, const std::vector<int32_t>& ci, const std::vector<double>& val,
                       cudaStream_t s);
    void pattern_outer(const std::vector<int64_t>& rp, const std::vector<int32_t>& ci, const std::vector<double>& val,
                       const double* d_u, const double* d_v, double alpha, double* d_out, cudaStream_t s);
    rsc_status pcg_batch(const std::vector<int64_t>& rp, const std::vector<int32_t>& ci, const std::vector<double>& val,
                         const std::vector<long long>& seg_ptr, const double* d_B, double* d_X, int nrhs, double rtol,
                         int max_iter, int* iters, double* relres, cudaStream_t s);
    rsc_status pcg(const std::vector<int64_t>& rp, const std::vector<int32_t>& ci, const std::vector<double>& val,
                   const double* d_b, double* d_x, double rtol, int max_iter, int* iters, double* relres,
                   cudaStream_t s);
    cudaStream_t stream = nullptr;
    DeviceMem amem;   // matrix for SpMV
    long long* d_rp = nullptr;
    int32_t* d_ci = nullptr;
    double* d_val = nullptr;
    bool a_uploaded = false;
    Scratch pcg_vec, red;
    double solve_seconds = 0.0;
    int last_iters = 0;
    double last_relres = 0.0;
    long long launches = 0;
};

// ------------------------------------------------------------------ PCG vector kernels (FP64)
__global__ void k_spmv(long long n, const long long* __restrict__ rp, const int32_t* __restrict__ ci,
                       const double* __restrict__ v, const double* __restrict__ x, double* __restrict__ y) {
    // 8 lanes per row
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    long long row = t >> 3;
    int sub = threadIdx.x & 7;
    double s = 0.0;
    if (row < n) {
        for (long long e = rp[row] + sub; e < rp[row + 1]; e += 8) s = fma(v[e], x[ci[e]], s);
    }
    for (int o = 4; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (row < n && sub == 0) y[row] = s;
}

// deterministic dot: per-block partials, then one block sums them in order
__global__ void k_dot_partial(long long n, const double* __restrict__ a, const double* __restrict__ b,
                              double* __restrict__ part) {
    double s = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        s = fma(a[i], b[i], s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ double ws[32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ws[w];
        part[blockIdx.x] = t;
    }
}
__global__ void k_dot_final(int nparts, const double* __restrict__ part, double* __restrict__ out) {
    __shared__ double ws[256];
    double s = 0.0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) s += part[i];
    ws[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) ws[threadIdx.x] += ws[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = ws[0];
}
// y = a*x + b*y
__global__ void k_axpby(long long n, double a, const double* __restrict__ x, double b, double* __restrict__ y) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = a * x[i] + b * y[i];
}
// y = x - y (residual from A x)
__global__ void k_xmy(long long n, const double* __restrict__ x, double* __restrict__ y) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = x[i] - y[i];
}

static constexpr int DOT_BLOCKS = 304;

// ------------------------------------------------------------------ batched PCG (systems x right-hand sides)
// Vectors are n x nrhs, column-major; a segment is one (system, column) pair, systems being
// contiguous row ranges seg_ptr[s] .. seg_ptr[s+1].  Pair index = column * nseg + system.
__global__ void k_spmv_multi(long long n, const long long* __restrict__ rp, const int32_t* __restrict__ ci,
                             const double* __restrict__ v, const double* __restrict__ X, double* __restrict__ Y) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long row = t >> 3;
    const int sub = threadIdx.x & 7;
    const double* x = X + (size_t)blockIdx.y * n;
    double s = 0.0;
    if (row < n)
        for (long long e = rp[row] + sub; e < rp[row + 1]; e += 8) s = fma(v[e], x[ci[e]], s);
    for (int o = 4; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (row < n && sub == 0) Y[(size_t)blockIdx.y * n + row] = s;
}
// out[pair] = <A, B> over the pair's segment: one CTA per pair, fixed reduction order
__global__ void k_seg_dot(long long n, int nseg, const long long* __restrict__ seg_ptr, const double* __restrict__ A,
                          const double* __restrict__ B, double* __restrict__ out) {
    const int sgi = blockIdx.x, col = blockIdx.y;
    const double* a = A + (size_t)col * n;
    const double* b = B + (size_t)col * n;
    double s = 0.0;
    for (long long i = seg_ptr[sgi] + threadIdx.x; i < seg_ptr[sgi + 1]; i += blockDim.x) s = fma(a[i], b[i], s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ double ws[8];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ws[w];
        out[(size_t)col * nseg + sgi] = t;
    }
}
// Y = a_pair X + b_pair Y over every column (coef arrays indexed by pair; nullptr = 1)
__global__ void k_seg_axpby(long long n, int nseg, const int32_t* __restrict__ seg_of, const double* __restrict__ a,
                            const double* __restrict__ X, const double* __restrict__ b, double* __restrict__ Y,
                            double sa, double sb) {
    const int col = blockIdx.y;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int pr = col * nseg + seg_of[i];
        const double ca = a ? sa * a[pr] : sa, cb = b ? sb * b[pr] : sb;
        const size_t k = (size_t)col * n + i;
        Y[k] = ca * X[k] + cb * Y[k];
    }
}

rsc_status EngineImpl::pcg_batch(const std::vector<int64_t>& rp, const std::vector<int32_t>& ci,
                                 const std::vector<double>& val, const std::vector<long long>& seg_ptr,
                                 const double* d_B, double* d_X, int nrhs, double rtol, int max_iter, int* iters,
                                 double* relres, cudaStream_t s) {
    const long long n = (long long)rp.size() - 1;
    const int nseg = (int)seg_ptr.size() - 1;
    const int np = nseg * nrhs;
    // the timed region starts before any host step of the solve (matrix upload, segment
    // tables, the N-column launch list)
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    CK(cudaEventRecord(e0, s));
    ensure_matrix(rp, ci, val, s);
    const size_t vbytes = sizeof(double) * (size_t)n * nrhs;
    char* W = (char*)pcg_vec.get(5 * vbytes + sizeof(double) * 8 * np + sizeof(long long) * (nseg + 1) +
                                 sizeof(int32_t) * n + 4096);
    double* R = (double*)W;
    double* Z = (double*)(W + vbytes);
    double* P = (double*)(W + 2 * vbytes);
    double* Q = (double*)(W + 3 * vbytes);
    double* T = (double*)(W + 4 * vbytes);
    double* sc = (double*)(W + 5 * vbytes);            // 8 np scalars
    long long* d_seg = (long long*)(sc + 8 * np);
    int32_t* d_segof = (int32_t*)(d_seg + nseg + 1);
    std::vector<int32_t> segof(n);
    for (int g = 0; g < nseg; ++g)
        for (long long i = seg_ptr[g]; i < seg_ptr[g + 1]; ++i) segof[i] = g;
    CK(cudaMemcpyAsync(d_seg, seg_ptr.data(), sizeof(long long) * (nseg + 1), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(d_segof, segof.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, s));
    const dim3 vg((unsigned)std::min(cdiv(n, 256), 2048), (unsigned)nrhs);
    auto seg_dot = [&](const double* A, const double* B, std::vector<double>& out) {
        k_seg_dot<<<dim3((unsigned)nseg, (unsigned)nrhs), 256, 0, s>>>(n, nseg, d_seg, A, B, sc);
        launches++;
        out.resize(np);
        CK(cudaMemcpyAsync(out.data(), sc, sizeof(double) * np, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    };
    auto put = [&](double* dst, const std::vector<double>& v) {
        CK(cudaMemcpyAsync(dst, v.data(), sizeof(double) * np, cudaMemcpyHostToDevice, s));
    };
    auto spmv = [&](const double* X, double* Y) {
        k_spmv_multi<<<dim3((unsigned)cdiv(n * 8, 256), (unsigned)nrhs), 256, 0, s>>>(n, d_rp, d_ci, d_val, X, Y);
        launches++;
    };
    auto precond = [&](const double* Rv, double* Zv) { apply_multi(Rv, Zv, nrhs, s); };
    prepare_multi(nrhs);   // the N-column launch list, built once per factorization
    double* d_alpha = sc + np;
    double* d_beta = sc + 2 * np;
    CK(cudaMemsetAsync(d_X, 0, vbytes, s));
    CK(cudaMemcpyAsync(R, d_B, vbytes, cudaMemcpyDeviceToDevice, s));
    std::vector<double> nb, rz, pq, rn, tr, alpha(np), beta(np);
    seg_dot(d_B, d_B, nb);
    for (auto& v : nb) v = std::sqrt(v);
    std::vector<char> active(np);
    for (int q = 0; q < np; ++q) {
        active[q] = nb[q] > 0.0;
        iters[q] = 0;
        relres[q] = 0.0;
    }
    precond(R, Z);
    CK(cudaMemcpyAsync(P, Z, vbytes, cudaMemcpyDeviceToDevice, s));
    seg_dot(R, Z, rz);
    int nact = 0;
    for (char a : active) nact += a;
    rsc_status st = RSC_OK;
    for (int it = 1; it <= max_iter && nact > 0; ++it) {
        spmv(P, Q);
        seg_dot(P, Q, pq);
        for (int q = 0; q < np; ++q) alpha[q] = active[q] ? rz[q] / pq[q] : 0.0;
        put(d_alpha, alpha);
        k_seg_axpby<<<vg, 256, 0, s>>>(n, nseg, d_segof, d_alpha, P, nullptr, d_X, 1.0, 1.0);
        k_seg_axpby<<<vg, 256, 0, s>>>(n, nseg, d_segof, d_alpha, Q, nullptr, R, -1.0, 1.0);
        launches += 2;
        seg_dot(R, R, rn);
        bool any = false;
        for (int q = 0; q < np; ++q) {
            if (!std::isfinite(rn[q])) { st = RSC_ERR_NOT_SPD; active[q] = 0; }
            else if (active[q] && std::sqrt(rn[q]) / nb[q] <= rtol) any = true;
        }
        if (any) {   // confirm with the true residual
            spmv(d_X, T);
            k_seg_axpby<<<vg, 256, 0, s>>>(n, nseg, d_segof, nullptr, d_B, nullptr, T, 1.0, -1.0);
            launches++;
            seg_dot(T, T, tr);
            for (int q = 0; q < np; ++q)
                if (active[q] && std::sqrt(rn[q]) / nb[q] <= rtol && std::sqrt(tr[q]) / nb[q] <= rtol) {
                    active[q] = 0;
                    iters[q] = it;
                    relres[q] = std::sqrt(tr[q]) / nb[q];
                }
        }
        nact = 0;
        for (int q = 0; q < np; ++q) {
            nact += active[q];
            if (active[q]) iters[q] = it;
        }
        if (nact == 0) break;
        precond(R, Z);
        std::vector<double> rz_new;
        seg_dot(R, Z, rz_new);
        for (int q = 0; q < np; ++q) beta[q] = active[q] ? rz_new[q] / rz[q] : 0.0;
        put(d_beta, beta);
        k_seg_axpby<<<vg, 256, 0, s>>>(n, nseg, d_segof, nullptr, Z, d_beta, P, 1.0, 1.0);
        launches++;
        rz = rz_new;
    }
    if (nact > 0) {
        spmv(d_X, T);
        k_seg_axpby<<<vg, 256, 0, s>>>(n, nseg, d_segof, nullptr, d_B, nullptr, T, 1.0, -1.0);
        seg_dot(T, T, tr);
        for (int q = 0; q < np; ++q)
            if (active[q]) relres[q] = nb[q] > 0 ? std::sqrt(tr[q]) / nb[q] : 0.0;
        if (st == RSC_OK) st = RSC_ERR_NO_CONVERGENCE;
    }
    CK(cudaEventRecord(e1, s));
    CK(cudaEventSynchronize(e1));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    solve_seconds = ms * 1e-3;
    int mx = 0;
    for (int q = 0; q < np; ++q) mx = std::max(mx, iters[q]);
    last_iters = mx;
    return st;
}

// out[e] = v[src[e]]
__global__ void k_gather_vals(const double* __restrict__ v, const long long* __restrict__ src, long long cnt,
                              double* __restrict__ out) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < cnt; e += (long long)gridDim.x * blockDim.x)
        out[e] = v[src[e]];
}

// out[e] = alpha * u[i] * v[j] for every stored entry e = (i, j) of the CSR pattern
__global__ void k_pattern_outer(long long n, const long long* __restrict__ rp, const int32_t* __restrict__ ci,
                                const double* __restrict__ u, const double* __restrict__ v, double alpha,
                                double* __restrict__ out) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long row = t >> 3;
    const int sub = threadIdx.x & 7;
    if (row >= n) return;
    const double ui = alpha * u[row];
    for (long long e = rp[row] + sub; e < rp[row + 1]; e += 8) out[e] = ui * v[ci[e]];
}

void EngineImpl::ensure_matrix(const std::vector<int64_t>& rp, const std::vector<int32_t>& ci,
                               const std::vector<double>& val, cudaStream_t s) {
    const long long n = (long long)rp.size() - 1;
    if (!a_uploaded) {   // cleared by values_changed()
        amem.release();
        d_rp = (long long*)amem.alloc(sizeof(long long) * (n + 1));
        CK(cudaMemcpyAsync(d_rp, rp.data(), sizeof(long long) * (n + 1), cudaMemcpyHostToDevice, s));
        d_ci = (int32_t*)amem.alloc(sizeof(int32_t) * ci.size());
        CK(cudaMemcpyAsync(d_ci, ci.data(), sizeof(int32_t) * ci.size(), cudaMemcpyHostToDevice, s));
        d_val = (double*)amem.alloc(sizeof(double) * val.size());
        if (vals_dev) CK(cudaMemcpyAsync(d_val, d_uval, sizeof(double) * val.size(), cudaMemcpyDeviceToDevice, s));
        else CK(cudaMemcpyAsync(d_val, val.data(), sizeof(double) * val.size(), cudaMemcpyHostToDevice, s));
        a_uploaded = true;
    }
}

// number of non-finite entries of v[0..n) (atomic count)
__global__ void k_count_nonfinite(const double* __restrict__ v, long long n, int* __restrict__ cnt) {
    int c = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        c += !isfinite(v[i]);
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(cnt, c);
}

void EngineImpl::set_values_device(const double* d_in, long long nnz, cudaStream_t s) {
    if (!d_uval || n_uval != nnz) {
        umem.release();
        d_uval = (double*)umem.alloc(sizeof(double) * (nnz + 2));
        n_uval = nnz;
    }
    int* d_cnt = (int*)(d_uval + nnz);   // 8 bytes past the values
    CK(cudaMemsetAsync(d_cnt, 0, sizeof(int), s));
    k_count_nonfinite<<<std::max(1, std::min(cdiv(nnz, 256), 1024)), 256, 0, s>>>(d_in, nnz, d_cnt);
    launches++;
    int bad = 0;
    CK(cudaMemcpyAsync(&bad, d_cnt, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (bad) throw Error(RSC_ERR_INVALID_ARG, "non-finite matrix value");
    CK(cudaMemcpyAsync(d_uval, d_in, sizeof(double) * nnz, cudaMemcpyDeviceToDevice, s));
    CK(cudaStreamSynchronize(s));   // the caller may reuse d_in on return; the engine's stream sees the copy
    vals_dev = true;
    a_uploaded = false;
}

void EngineImpl::pattern_outer(const std::vector<int64_t>& rp, const std::vector<int32_t>& ci,
                               const std::vector<double>& val, const double* d_u, const double* d_v, double alpha,
                               double* d_out, cudaStream_t s) {
    const long long n = (long long)rp.size() - 1;
    ensure_matrix(rp, ci, val, s);
    k_pattern_outer<<<cdiv(n * 8, 256), 256, 0, s>>>(n, d_rp, d_ci, d_u, d_v, alpha, d_out);
    launches++;
    CK(cudaGetLastError());
}

rsc_status EngineImpl::pcg(const std::vector<int64_t>& rp, const std::vector<int32_t>& ci,
                           const std::vector<double>& val, const double* d_b, double* d_x, double rtol, int max_iter,
                           int* iters_out, double* relres_out, cudaStream_t s) {
    const long long n = (long long)rp.size() - 1;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    CK(cudaEventRecord(e0, s));   // the matrix upload (when values changed) is part of the solve
    ensure_matrix(rp, ci, val, s);
    double* V = (double*)pcg_vec.get(sizeof(double) * 5 * n);
    double *r = V, *z = V + n, *p = V + 2 * n, *q = V + 3 * n, *t = V + 4 * n;
    double* part = (double*)red.get(sizeof(double) * (DOT_BLOCKS + 8));
    double* scal = part + DOT_BLOCKS;
    double h_s[4];
    auto dot = [&](const double* a, const double* b) -> double {
        PROF(prof, "dot", s, 2.0 * n, 16.0 * n, k_dot_partial<<<DOT_BLOCKS, 256, 0, s>>>(n, a, b, part);
             k_dot_final<<<1, 256, 0, s>>>(DOT_BLOCKS, part, scal));
        launches += 2;
        CK(cudaMemcpyAsync(h_s, scal, sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        return h_s[0];
    };
    const int vb = (int)std::min<long long>(cdiv(n, 256), 4 * 152);
    auto spmv = [&](const double* x, double* y) {
        const double nnz = (double)val.size();
        PROF(prof, "spmv", s, 2.0 * nnz, 12.0 * nnz + 8.0 * (n + 1) + 16.0 * n,
             k_spmv<<<cdiv(n * 8, 256), 256, 0, s>>>(n, d_rp, d_ci, d_val, x, y));
        launches++;
    };
    CK(cudaMemsetAsync(d_x, 0, sizeof(double) * n, s));
    CK(cudaMemcpyAsync(r, d_b, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    const double nb = std::sqrt(dot(d_b, d_b));
    rsc_status st = RSC_OK;
    int it = 0;
    double rel = 0.0;
    if (nb == 0.0) {
        rel = 0.0;
    } else {
        apply(r, z, s);
        CK(cudaMemcpyAsync(p, z, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
        double rz = dot(r, z);
        bool done = false;
        for (it = 1; it <= max_iter; ++it) {
            spmv(p, q);
            const double pq = dot(p, q);
            const double alpha = rz / pq;
            PROF(prof, "axpy", s, 6.0 * n, 48.0 * n, k_axpby<<<vb, 256, 0, s>>>(n, alpha, p, 1.0, d_x);
                 k_axpby<<<vb, 256, 0, s>>>(n, -alpha, q, 1.0, r));
            launches += 2;
            const double rn = std::sqrt(dot(r, r));
            if (!std::isfinite(rn)) { st = RSC_ERR_NOT_SPD; break; }
            if (rn / nb <= rtol) {
                spmv(d_x, t);
                k_xmy<<<vb, 256, 0, s>>>(n, d_b, t);
                launches++;
                rel = std::sqrt(dot(t, t)) / nb;
                if (rel <= rtol) { done = true; break; }
            }
            apply(r, z, s);
            const double rz_new = dot(r, z);
            const double beta = rz_new / rz;
            rz = rz_new;
            PROF(prof, "axpy", s, 3.0 * n, 24.0 * n, k_axpby<<<vb, 256, 0, s>>>(n, 1.0, z, beta, p));
            launches++;
        }
        if (!done) {
            if (it > max_iter) it = max_iter;
            spmv(d_x, t);
            k_xmy<<<vb, 256, 0, s>>>(n, d_b, t);
            launches++;
            rel = std::sqrt(dot(t, t)) / nb;
            if (st == RSC_OK) st = RSC_ERR_NO_CONVERGENCE;
        }
    }
    CK(cudaEventRecord(e1, s));
    CK(cudaEventSynchronize(e1));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    solve_seconds = ms * 1e-3;
    prof.flush();
    last_iters = it;
    last_relres = rel;
    if (iters_out) *iters_out = it;
    if (relres_out) *relres_out = rel;
    return st;
}

// ------------------------------------------------------------------ typed engine
// Section 5.1: one sparse factor of the interior-block products, A restricted to a row set
// (CSR rows listed compactly; CSR row i is row rmap[i] of the product's output).
struct IbCsr { CsrBlock blk{}; const int32_t* rmap = nullptr; int pend = -1; long long moff = 0; };   // pend, moff: plan-time bookkeeping
// The Eq. interiorBlockMult term of interior block b in the products with a block of L:
// f (L X): t = A(C_B, cols) X, W(rows) -= A(rows, C_B) L_B^{-T} L_B^{-1} t; t (L^T G) the same with
// rows and columns exchanged.
struct IbTerm { int b = 0; IbCsr in_f, out_f, in_t, out_t; };

template <class T>
struct EngineT final : EngineImpl {
    struct NodeRT {
        int c = 0, r = 0;
        long long c0 = 0;
        bool compressed = false, hier = false;
        long long off = -1;     // panel or dense-diagonal offset in the arena
        int ld = 0;
        std::vector<long long> leaf_off;   // by block label (leaves only)
        long long inv_off = -1;            // row-major inverses of the SOLVE_MAX diagonal sub-blocks
        std::vector<long long> leaf_inv;   // by label: row-major inverse of each leaf
        int rank = 0;
        T* V = nullptr;          // |R_j| x rank, column-major
        T* U = nullptr;          // c x rank, column-major (ld c)
        std::vector<int> brank;            // by label
        std::vector<T*> bV, bU;
        // factors of the off-diagonal blocks of the inverse, by label (internal blocks):
        // (L^D)^{-1} holds -tV_s tU_s^T in the place of V_s U_s^T, with tV_s = L_right(s)^{-1} V_s
        // and tU_s = L_left(s)^{-T} U_s (same shapes as V_s, U_s)
        std::vector<T*> tV, tU;
        // sparse A blocks for the implicit products (compressed nodes)
        CsrBlock aR{}, aC{};               // A(R_j, C_j) by R rows / by C rows (transposed)
        std::vector<CsrBlock> bR, bC;      // per internal block: A(rows_s, cols_s) by rows / by cols
        int32_t* tailpos = nullptr;        // per descendant: positions of R_k's tail rows inside R_j
        std::vector<long long> tail_off;   // offset of descendant d's tail map inside tailpos
        int ib = -1;                       // interior block holding this supernode (Section 5.1), -1: none
        std::vector<std::vector<IbTerm>> ibt;   // by label (0: L^O_j): interior-block terms
    };

    const Symbolic& S;
    rsc_options o;
    DeviceMem pmem;      // plan (per layout)
    DeviceMem fmem;      // factor arena + low-rank storage
    T* arena = nullptr;
    long long arena_elems = 0;
    T* invs = nullptr;            // inverses of dense diagonal (sub-)blocks, row-major
    long long inv_elems = 0;
    std::vector<TrsvTask*> inv_tasks;   // per level: inverse computations of the level's dense blocks
    std::vector<int> inv_count, inv_maxc;
    // inverse of the b-th SOLVE_MAX diagonal sub-block of a non-hierarchical node
    const T* inv_block(int j, int b0) const {
        const NodeRT& n = nd[j];
        long long o = n.inv_off;
        for (int x = 0; x < b0; x += SOLVE_MAX) { const long long bs = std::min(SOLVE_MAX, n.c - x); o += bs * bs; }
        return invs + o;
    }
    std::vector<TrsvTask> inverse_tasks_dense(int j) const {
        const NodeRT& n = nd[j];
        std::vector<TrsvTask> v;
        for (int b0 = 0; b0 < n.c; b0 += SOLVE_MAX) {
            const int bs = std::min(SOLVE_MAX, n.c - b0);
            v.push_back(TrsvTask{arena + n.off + b0 + (size_t)b0 * n.ld, n.ld, bs, bs, (void*)inv_block(j, b0), bs, 2});
        }
        return v;
    }
    void launch_inverses(std::vector<TrsvTask>& tv, const TrsvTask* dev = nullptr) {
        if (tv.empty()) return;
        int maxc = 0;
        for (auto& t : tv) maxc = std::max(maxc, t.c);
        const TrsvTask* d = dev ? dev : (const TrsvTask*)upload_tmp(sTask, tv);
        const dim3 grid((unsigned)tv.size(), (unsigned)cdiv(maxc, TRSV_CW));
        double fl = 0;
        for (auto& t : tv) fl += (double)t.c * t.c * t.c / 3.0;
        flops += fl;
        PROF(prof, "trinv", stream, fl, 0, k_trsv_subst<T, TRSV_CW><<<grid, 256, 0, stream>>>(d));
        launches++;
        LAUNCH_CHECK();
    }
    T* lr_base = nullptr;
    long long lr_cap = 0, lr_used = 0;
    std::vector<NodeRT> nd;

    // ---------------------------------------------------------------- interior blocks (Section 5.1)
    // A maximal subtree of the supernodal tree without a compressed supernode; its supernodes are
    // the contiguous run first..last (postorder) and its columns C_B = [c0, c1).  Their panels keep
    // the rows inside C_B only: those rows are the sparse factor L_B = chol(A(C_B, C_B)) (Eq.
    // interiorDiagonalDef); L(R_B, C_B) is never formed, its uses go through A(., C_B) L_B^{-T}
    // (Eqs. interiorBlockClosedForm, interiorBlockMult).
    struct IbEntry { int32_t x, y; long long src; };   // A(x, c0 + y), x outside C_B (x >= c1)
    struct IBlock {
        int first = 0, last = 0, root_level = 0;
        long long c0 = 0, c1 = 0;
        std::vector<std::vector<int>> lvl;   // the block's supernodes by level (0 .. root_level)
        std::vector<IbEntry> adj;            // sorted by (x, y)
        IbCsr fwd, bwd;                      // apply: A(R_B, C_B) by rows x, A(C_B, R_B) by rows y (global)
    };
    // A dense target region (a dense diagonal, a diagonal leaf or an uncompressed panel outside
    // every block) receiving block b's Schur complement C(P, Q) = A(P, C_B) A_BB^{-1} A(C_B, Q):
    // in = A(C_B, P) (CSR columns index P), out = A(Q, C_B) with rmap = column positions of Q in the
    // region, cmap = row positions of P; the region is column-major at base with leading dim ld.
    struct IbDense { int b = 0; T* base = nullptr; int ld = 0; int nP = 0; IbCsr in, out; const int32_t* cmap = nullptr; long long cmoff = 0; };
    std::vector<IBlock> iblocks;
    std::vector<std::vector<int>> ib_root;          // by level: blocks whose root is at that level
    std::vector<std::vector<IbDense>> ib_dense;     // by level of the block root
    bool ib_on = false;
    int ib_maxP = 0;
    T* ib_win = nullptr;     // (2 ib_maxP + 64) x 64, rows ib_maxP .. ib_maxP + 63 the identity
    T* d_zero = nullptr;     // one zero (source of zero fills)

    // blocks of the current plan; truncates the rows of their supernodes to those inside C_B
    void find_interior_blocks() {
        iblocks.clear();
        ib_root.assign(S.nlevels, {});
        ib_on = o.interior_blocks != 0;
        if (!ib_on) return;
        const int M = S.M;
        std::vector<char> bad(M);
        std::vector<int> first(M);
        for (int j = 0; j < M; ++j) { bad[j] = nd[j].compressed; first[j] = j; }
        for (int j = 0; j < M; ++j) {   // children precede their parents
            const int p = S.parent[j];
            if (p >= 0) {
                if (p <= j) throw Error(RSC_ERR_INVALID_ARG, "supernodes not in postorder");
                bad[p] = bad[p] || bad[j];
                first[p] = std::min(first[p], first[j]);
            }
        }
        for (int j = 0; j < M; ++j) {
            const int p = S.parent[j];
            if (bad[j] || (p >= 0 && !bad[p])) continue;   // not the root of a maximal clean subtree
            IBlock B;
            B.first = first[j];
            B.last = j;
            B.c0 = S.sn_ptr[first[j]];
            B.c1 = S.sn_ptr[j + 1];
            B.root_level = S.level[j];
            B.lvl.assign(B.root_level + 1, {});
            for (int k = B.first; k <= j; ++k) {
                if (bad[k] || S.level[k] > B.root_level) throw Error(RSC_ERR_INVALID_ARG, "interior block not contiguous");
                nd[k].ib = (int)iblocks.size();
                B.lvl[S.level[k]].push_back(k);
                const int32_t* Rk = S.R(k);
                nd[k].r = (int)(std::lower_bound(Rk, Rk + S.nrows(k), (int32_t)B.c1) - Rk);
            }
            ib_root[B.root_level].push_back((int)iblocks.size());
            iblocks.push_back(std::move(B));
        }
    }
    bool plan_compress = false, plan_diag = false, have_plan = false;
    bool is_factored = false;
    double tol = 0.0, tol_D = 0.0;
    bool fixed = false;          // Section 5.2 ranks instead of the adaptive stopping test
    FixedRank fr_cur;            // alpha_D as grown by the restarts of this factorization
    int restarts = 0;
    bool diag_on = false;
    // device tables
    int32_t* d_rows = nullptr;
    long long* d_rows_ptr = nullptr;
    int32_t* d_perm = nullptr;
    NodeTgt* d_tgt = nullptr;
    LeafMap* d_leaf = nullptr;
    LoOp* d_lo = nullptr;
    std::vector<LoOp> h_lo;
    long long* d_asm_src = nullptr;
    long long* d_asm_dst = nullptr;
    long long asm_cnt = 0;
    double* d_valbuf = nullptr;
    int* d_status = nullptr;
    // arrival counters of row-split TN products; every counter is back at zero when the
    // launch that used it ends, so each launch numbers its counters from 0
    static constexpr int TN_CNT_CAP = 1 << 16;
    static constexpr int TN_SPLIT_MIN = 512, TN_SPLIT_ROWS = 256, TN_SPLIT_MAX = 64;
    static constexpr int TN1_SPLIT_ROWS = 512;   // rows per CTA of a split vector TN task (apply)
    unsigned* d_tncnt = nullptr;
    double* d_norms = nullptr;     // [0] y1, [1] current
    double* d_small = nullptr;     // gram (256) + rinv (256)
    int* d_qstatus = nullptr;
    // per level task lists
    struct PanelStep { PotrfTask* potrf; int npotrf; TrsmTask* trsm; int ntrsm; GemmTask* gemm; int ngemm;
                       double fl_potrf, fl_trsm, fl_gemm; };
    struct PushElems { int k; double elems; double rows; };
    std::vector<std::vector<PushElems>> push_elems;   // per level: per source, lower entries pushed
    std::vector<std::vector<PanelStep>> panel_steps;   // [level][step]
    std::vector<PushTask*> push_tasks;
    std::vector<int> push_count;
    bool tc = false;                      // BF16 / TF32 forms: extend-add on tcgen05 tensor cores
    bool tc_tf32 = false;                 // TF32 operands (kind::tf32) instead of BF16
    std::vector<PushTask*> push_tasks_tc; // 128 x 64 tiles
    std::vector<int> push_count_tc;
    // sparse block values are gathered at factor time from these source indices
    std::vector<long long> sp_src;     // concatenated value sources of all CsrBlocks
    double* d_spval = nullptr;
    long long* d_spsrc = nullptr;
    // scratch
    Scratch sG, sY, sUr, sVr, sX, sZ, sT, sTv, sTask, sTask2, sT2;
    double flops = 0.0;
    double factor_seconds = 0.0;
    // solve scratch
    Scratch sy, stmp;

    EngineT(const Symbolic& S_, const rsc_options& o_) : S(S_), o(o_) {
        tc = sizeof(T) == 4 && (o.precision == RSC_PREC_BF16 || o.precision == RSC_PREC_TF32);
        tc_tf32 = tc && o.precision == RSC_PREC_TF32;
        CK(cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking));
        if (tc) {
            CK(cudaFuncSetAttribute(k_push_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_PAD_SMEM));
            CK(cudaFuncSetAttribute(k_push_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_PAD_SMEM_TF32));
            if (tc_tf32) tc_attrs<true>(); else tc_attrs<false>();
        }
        CK(cudaFuncSetAttribute(k_leaf_factor<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)LEAF_SMEM_CAP));
        CK(cudaFuncSetAttribute(k_tn_s<T, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ts_smem_bytes<T>(16)));
        CK(cudaFuncSetAttribute(k_tn_s<T, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ts_smem_bytes<T>(32)));
        CK(cudaFuncSetAttribute(k_tn_s<T, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ts_smem_bytes<T>(64)));
        CK(cudaFuncSetAttribute(k_rf_dense<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)RFD_SMEM_CAP));
        CK(cudaFuncSetAttribute(k_trsv_tile<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tt_smem_bytes<T>()));
        if (const char* e = std::getenv("RSC_PROFILE")) { prof.on = true; if (std::strcmp(e, "1") != 0) prof.only = e; }
        hs_attr<8>();
        hs_attr<4>();
        hs_attr<2>();
        hs_attr<1>();
        nd.resize(S.M);
    }
    ~EngineT() override {
        if (dense_graph) cudaGraphExecDestroy(dense_graph);
        plan1.clear();
        planN.clear();
        if (arena_base) cudaFree(arena_base);
        if (arena_host) cudaFreeHost(arena_host);
        if (rf_host) cudaFreeHost(rf_host);
        if (rank_host) cudaFreeHost(rank_host);
        if (d_rfp_time) cudaFree(d_rfp_time);
        if (st_host) cudaFreeHost(st_host);
        if (stream) cudaStreamDestroy(stream);
    }

    bool factored() const override { return is_factored; }

    // ---------------------------------------------------------------- plan
    void build_plan(bool compress, bool diag) {
        pmem.release();
        fmem.release();
        have_plan = false;
        const int M = S.M;
        long long off = 0;
        for (int j = 0; j < M; ++j) {
            NodeRT& n = nd[j];
            n = NodeRT();
            n.c = S.ncols(j);
            n.r = S.nrows(j);
            n.c0 = S.sn_ptr[j];
            n.compressed = compress && S.kind[j] == 1 && n.c >= o.tau_O;
            n.hier = n.compressed && diag && S.tree[j].nblocks > 0;
        }
        find_interior_blocks();
        for (int j = 0; j < M; ++j) {
            NodeRT& n = nd[j];
            if (!n.compressed) {
                n.off = off;
                n.ld = n.c + n.r;
                off += (long long)n.ld * n.c;
            } else if (!n.hier) {
                n.off = off;
                n.ld = n.c;
                off += (long long)n.c * n.c;
            } else {
                const BlockTree& t = S.tree[j];
                n.leaf_off.assign(t.nblocks + 1, -1);
                for (int s = 1; s <= t.nblocks; ++s)
                    if (t.leaf[s]) {
                        long long sz = t.hi[s] - t.lo[s];
                        n.leaf_off[s] = off;
                        off += sz * sz;
                    }
                n.brank.assign(t.nblocks + 1, 0);
                n.bV.assign(t.nblocks + 1, nullptr);
                n.bU.assign(t.nblocks + 1, nullptr);
                n.tV.assign(t.nblocks + 1, nullptr);
                n.tU.assign(t.nblocks + 1, nullptr);
            }
        }
        arena_elems = off;
        arena = (T*)fmem.alloc(sizeof(T) * std::max<long long>(off, 1));
        long long ioff = 0;
        for (int j = 0; j < M; ++j) {
            NodeRT& n = nd[j];
            if (!n.hier) {
                n.inv_off = ioff;
                for (int b0 = 0; b0 < n.c; b0 += SOLVE_MAX) {
                    const long long bs = std::min(SOLVE_MAX, n.c - b0);
                    ioff += bs * bs;
                }
            } else {
                const BlockTree& t = S.tree[j];
                n.leaf_inv.assign(t.nblocks + 1, -1);
                for (int b = 1; b <= t.nblocks; ++b)
                    if (t.leaf[b]) {
                        const long long sz = t.hi[b] - t.lo[b];
                        n.leaf_inv[b] = ioff;
                        ioff += sz * sz;
                    }
            }
        }
        invs = (T*)fmem.alloc(sizeof(T) * std::max<long long>(ioff, 1));
        inv_elems = ioff;
        // low-rank storage bound: U (c x maxr) + V (r x maxr) per compressed block
        long long lr = 0;
        for (int j = 0; j < M; ++j) {
            const NodeRT& n = nd[j];
            if (!n.compressed) continue;
            long long mr = std::min(n.c, n.r);
            lr += (long long)(n.c + n.r) * mr + 64;
            if (n.hier) {
                const BlockTree& t = S.tree[j];
                for (int s = 1; s <= t.nblocks; ++s)
                    if (!t.leaf[s]) {
                        long long a = t.hi[s] - t.mid[s], b = t.mid[s] - t.lo[s];
                        lr += 2 * ((a + b) * std::min(a, b) + 64);   // V_s, U_s and tV_s, tU_s
                    }
            }
        }
        lr_cap = lr;
        lr_base = (T*)fmem.alloc(sizeof(T) * std::max<long long>(lr, 1));

        // device structure tables
        d_rows = pmem.upload(S.rows, stream);
        std::vector<long long> rptr(S.rows_ptr.begin(), S.rows_ptr.end());
        d_rows_ptr = pmem.upload(rptr, stream);
        d_perm = pmem.upload(S.perm, stream);
        d_status = (int*)pmem.alloc(sizeof(int) * 4);
        d_tncnt = (unsigned*)pmem.alloc(sizeof(unsigned) * TN_CNT_CAP);
        CK(cudaMemsetAsync(d_tncnt, 0, sizeof(unsigned) * TN_CNT_CAP, stream));
        d_rfbar = (RfBarrier*)pmem.alloc(sizeof(RfBarrier));
        CK(cudaMemsetAsync(d_rfbar, 0, sizeof(RfBarrier), stream));
        d_norms = (double*)pmem.alloc(sizeof(double) * 4);
        d_small = (double*)pmem.alloc(sizeof(double) * 512);
        d_qstatus = (int*)pmem.alloc(sizeof(int) * 4);

        // targets and leaf maps
        std::vector<NodeTgt> tg(M);
        std::vector<LeafMap> lm(S.n, LeafMap{0, 0, 0, 0});
        for (int j = 0; j < M; ++j) {
            const NodeRT& n = nd[j];
            NodeTgt t{};
            t.c = n.c;
            t.r = n.r;
            t.c0 = n.c0;
            t.rows_off = S.rows_ptr[j];
            if (!n.compressed) { t.kind = 0; t.base = arena + n.off; t.ld = n.ld; }
            else if (!n.hier) { t.kind = 1; t.base = arena + n.off; t.ld = n.c; }
            else {
                t.kind = 2;
                t.base = nullptr;
                t.ld = 0;
                const BlockTree& bt = S.tree[j];
                for (int s = 1; s <= bt.nblocks; ++s)
                    if (bt.leaf[s])
                        for (int q = bt.lo[s]; q < bt.hi[s]; ++q)
                            lm[n.c0 + q] = LeafMap{n.c0 + bt.lo[s], n.leaf_off[s], bt.hi[s] - bt.lo[s], 0};
            }
            tg[j] = t;
        }
        d_tgt = pmem.upload(tg, stream);
        d_leaf = pmem.upload(lm, stream);
        h_lo.assign(M, LoOp{nullptr, 1, 0});
        for (int j = 0; j < M; ++j)
            if (!nd[j].compressed) h_lo[j] = LoOp{arena + nd[j].off + nd[j].c, nd[j].ld, nd[j].c};
        d_lo = (LoOp*)pmem.alloc(sizeof(LoOp) * M);

        // assembly map and sparse blocks
        std::vector<long long> src, dst;
        src.reserve(S.li.size());
        dst.reserve(S.li.size());
        sp_src.clear();
        struct Coo { int r, c; long long s; };
        std::vector<std::vector<Coo>> offA(M);
        std::vector<std::vector<std::vector<Coo>>> blkA(M);
        for (int j = 0; j < M; ++j)
            if (nd[j].hier) blkA[j].assign(S.tree[j].nblocks + 1, {});
        for (long long c = 0; c < S.n; ++c) {
            const int j = S.snode_of[c];
            const NodeRT& n = nd[j];
            const int lc = (int)(c - n.c0);
            const int32_t* Rj = S.R(j);
            const long long bc1 = n.ib >= 0 ? iblocks[n.ib].c1 : S.n;
            for (long long e = S.lp[c]; e < S.lp[c + 1]; ++e) {
                const long long g = S.li[e];
                if (g >= bc1) {   // A(R_B, C_B): kept sparse for the closed forms
                    IBlock& B = iblocks[n.ib];
                    B.adj.push_back(IbEntry{(int32_t)g, (int32_t)(c - B.c0), S.lsrc[e]});
                    continue;
                }
                const bool inC = g < n.c0 + n.c;
                const int lr = inC ? (int)(g - n.c0) : (int)(std::lower_bound(Rj, Rj + n.r, (int32_t)g) - Rj);
                if (!n.compressed) {
                    src.push_back(S.lsrc[e]);
                    dst.push_back(n.off + (inC ? lr : n.c + lr) + (long long)lc * n.ld);
                } else if (!inC) {
                    offA[j].push_back({lr, lc, S.lsrc[e]});
                } else if (!n.hier) {
                    src.push_back(S.lsrc[e]);
                    dst.push_back(n.off + lr + (long long)lc * n.c);
                } else {
                    const BlockTree& bt = S.tree[j];
                    int s = bt.root;
                    while (!bt.leaf[s]) {
                        if (lc < bt.mid[s] && lr >= bt.mid[s]) break;
                        s = lr < bt.mid[s] ? bt.left[s] : bt.right[s];
                    }
                    if (bt.leaf[s]) {
                        const long long sz = bt.hi[s] - bt.lo[s];
                        src.push_back(S.lsrc[e]);
                        dst.push_back(n.leaf_off[s] + (lr - bt.lo[s]) + (lc - bt.lo[s]) * sz);
                    } else {
                        blkA[j][s].push_back({lr - bt.mid[s], lc - bt.lo[s], S.lsrc[e]});
                    }
                }
            }
        }
        asm_cnt = (long long)src.size();
        d_asm_src = pmem.upload(src, stream);
        d_asm_dst = pmem.upload(dst, stream);
        d_valbuf = (double*)pmem.alloc(sizeof(double) * (S.lsrc.empty() ? 1 : (size_t)(*std::max_element(S.lsrc.begin(), S.lsrc.end()) + 1)));

        // CSR blocks (two orientations); values gathered per factor via sp_src
        std::vector<int32_t> sp_rp, sp_ci;
        struct PendingBlk { int node, label, orient; long long rp_off, ci_off, v_off; int nrows; };
        std::vector<PendingBlk> pend;
        auto add_csr = [&](std::vector<Coo>& coo, int nrows, bool by_row, int node, int label) {
            std::vector<int> cnt(nrows + 1, 0);
            for (auto& x : coo) cnt[(by_row ? x.r : x.c) + 1]++;
            for (int i = 0; i < nrows; ++i) cnt[i + 1] += cnt[i];
            PendingBlk pb{node, label, by_row ? 0 : 1, (long long)sp_rp.size(), (long long)sp_ci.size(),
                          (long long)sp_src.size(), nrows};
            std::vector<int> fill(cnt.begin(), cnt.end() - 1);
            std::vector<int32_t> col(coo.size());
            std::vector<long long> sv(coo.size());
            // stable order: sort by (row, col)
            std::vector<size_t> idx(coo.size());
            std::iota(idx.begin(), idx.end(), 0);
            std::sort(idx.begin(), idx.end(), [&](size_t a, size_t b) {
                int ra = by_row ? coo[a].r : coo[a].c, rb = by_row ? coo[b].r : coo[b].c;
                int ca = by_row ? coo[a].c : coo[a].r, cb = by_row ? coo[b].c : coo[b].r;
                return ra != rb ? ra < rb : ca < cb;
            });
            for (size_t t = 0; t < idx.size(); ++t) {
                const Coo& x = coo[idx[t]];
                col[t] = by_row ? x.c : x.r;
                sv[t] = x.s;
            }
            sp_rp.insert(sp_rp.end(), cnt.begin(), cnt.end());
            sp_ci.insert(sp_ci.end(), col.begin(), col.end());
            sp_src.insert(sp_src.end(), sv.begin(), sv.end());
            pend.push_back(pb);
        };
        for (int j = 0; j < M; ++j) {
            NodeRT& n = nd[j];
            if (!n.compressed) continue;
            add_csr(offA[j], n.r, true, j, 0);
            add_csr(offA[j], n.c, false, j, 0);
            if (n.hier) {
                const BlockTree& bt = S.tree[j];
                n.bR.assign(bt.nblocks + 1, CsrBlock{});
                n.bC.assign(bt.nblocks + 1, CsrBlock{});
                for (int s = 1; s <= bt.nblocks; ++s)
                    if (!bt.leaf[s]) {
                        add_csr(blkA[j][s], bt.hi[s] - bt.mid[s], true, j, s);
                        add_csr(blkA[j][s], bt.mid[s] - bt.lo[s], false, j, s);
                    }
            }
        }
        // interior blocks (Section 5.1): sparse factors of the closed forms, rows listed compactly
        std::vector<int32_t> ibmap;
        ib_dense.assign(S.nlevels, {});
        ib_maxP = 0;
        if (ib_on) {
            struct Ent { long long key; int col; long long src; };
            // CSR over the distinct keys (ascending); CSR row i is output row keymap(key_i)
            auto ib_build = [&](std::vector<Ent>& ent, auto keymap, IbCsr& dst) {
                std::sort(ent.begin(), ent.end(), [](const Ent& a, const Ent& b) {
                    return a.key != b.key ? a.key < b.key : a.col < b.col;
                });
                std::vector<Coo> coo;
                std::vector<int32_t> rm;
                long long last = -1;
                for (const Ent& e : ent) {
                    if (rm.empty() || e.key != last) { rm.push_back((int32_t)keymap(e.key)); last = e.key; }
                    coo.push_back(Coo{(int)rm.size() - 1, e.col, e.src});
                }
                dst.pend = (int)pend.size();
                add_csr(coo, (int)rm.size(), true, -1, 0);
                dst.moff = (long long)ibmap.size();
                ibmap.insert(ibmap.end(), rm.begin(), rm.end());
            };
            auto ident = [](long long k) { return k; };
            for (IBlock& B : iblocks) {
                std::sort(B.adj.begin(), B.adj.end(), [](const IbEntry& a, const IbEntry& b) {
                    return a.x != b.x ? a.x < b.x : a.y < b.y;
                });
                std::vector<Ent> f, bw;
                for (const IbEntry& e : B.adj) {
                    f.push_back(Ent{e.x, (int)(B.c0 + e.y), e.src});
                    bw.push_back(Ent{e.y, e.x, e.src});
                }
                const long long c0 = B.c0;
                ib_build(f, ident, B.fwd);
                ib_build(bw, [c0](long long k) { return c0 + k; }, B.bwd);
            }
            // entries of block B with x in the global range [g0, g1)
            auto in_range = [](const IBlock& B, long long g0, long long g1) {
                auto lo = std::lower_bound(B.adj.begin(), B.adj.end(), g0,
                                           [](const IbEntry& e, long long g) { return (long long)e.x < g; });
                auto hi = std::lower_bound(lo, B.adj.end(), g1,
                                           [](const IbEntry& e, long long g) { return (long long)e.x < g; });
                return std::make_pair(lo, hi);
            };
            // Eq. interiorBlockMult terms of the compressed supernodes
            for (int j = 0; j < M; ++j) {
                NodeRT& n = nd[j];
                if (!n.compressed) continue;
                std::vector<int> bl;
                for (long long d = S.desc_ptr[j]; d < S.desc_ptr[j + 1]; ++d)
                    if (nd[S.desc_k[d]].ib >= 0) bl.push_back(nd[S.desc_k[d]].ib);
                std::sort(bl.begin(), bl.end());
                bl.erase(std::unique(bl.begin(), bl.end()), bl.end());
                if (bl.empty()) continue;
                const BlockTree& bt = S.tree[j];
                const int nlab = n.hier ? bt.nblocks : 0;
                n.ibt.assign(nlab + 1, {});
                const int32_t* Rj = S.R(j);
                for (int b : bl) {
                    const IBlock& B = iblocks[b];
                    auto rc = in_range(B, n.c0, n.c0 + n.c);
                    std::vector<IbEntry> inC(rc.first, rc.second), inR;
                    for (const IbEntry& e : B.adj) {
                        if (e.x < n.c0 + n.c) continue;
                        const int pos = (int)(std::lower_bound(Rj, Rj + n.r, e.x) - Rj);
                        if (pos < n.r && Rj[pos] == e.x) inR.push_back(IbEntry{pos, e.y, e.src});
                    }
                    for (IbEntry& e : inC) e.x -= (int32_t)n.c0;   // local to C_j
                    // rows / columns of the block of L the product is taken with: (X in ro, C_B), (X in co, C_B)
                    auto term = [&](const std::vector<IbEntry>& ro, const std::vector<IbEntry>& co, int rbase, int cbase,
                                    std::vector<IbTerm>& dst) {
                        if (ro.empty() || co.empty()) return;
                        IbTerm tm;
                        tm.b = b;
                        std::vector<Ent> e1, e2, e3, e4;
                        for (const IbEntry& e : co) {
                            e1.push_back(Ent{e.y, e.x - cbase, e.src});    // in_f: t = A(C_B, cols) X
                            e4.push_back(Ent{e.x - cbase, e.y, e.src});    // out_t: W(cols) -= A(cols, C_B) t
                        }
                        for (const IbEntry& e : ro) {
                            e2.push_back(Ent{e.x - rbase, e.y, e.src});    // out_f: W(rows) -= A(rows, C_B) t
                            e3.push_back(Ent{e.y, e.x - rbase, e.src});    // in_t: t = A(C_B, rows) G
                        }
                        ib_build(e1, ident, tm.in_f);
                        ib_build(e2, ident, tm.out_f);
                        ib_build(e3, ident, tm.in_t);
                        ib_build(e4, ident, tm.out_t);
                        dst.push_back(tm);
                    };
                    term(inR, inC, 0, 0, n.ibt[0]);   // L^O_j: rows R_j, columns C_j
                    for (int sl = 1; sl <= nlab; ++sl) {
                        if (bt.leaf[sl]) continue;
                        std::vector<IbEntry> ro, co;
                        for (const IbEntry& e : inC) {
                            if (e.x >= bt.mid[sl] && e.x < bt.hi[sl]) ro.push_back(e);
                            if (e.x >= bt.lo[sl] && e.x < bt.mid[sl]) co.push_back(e);
                        }
                        term(ro, co, bt.mid[sl], bt.lo[sl], n.ibt[sl]);
                    }
                }
            }
            // dense targets of each block's Schur complement
            for (int b = 0; b < (int)iblocks.size(); ++b) {
                const IBlock& B = iblocks[b];
                std::vector<int> tj;
                for (const IbEntry& e : B.adj) tj.push_back(S.snode_of[e.x]);
                std::sort(tj.begin(), tj.end());
                tj.erase(std::unique(tj.begin(), tj.end()), tj.end());
                // P: (storage row position, entry), Q: (storage column position, entry)
                auto region = [&](std::vector<std::pair<int, IbEntry>>& P, std::vector<std::pair<int, IbEntry>>& Q, T* base,
                                  int ld) {
                    if (P.empty() || Q.empty()) return;
                    IbDense dn;
                    dn.b = b;
                    dn.base = base;
                    dn.ld = ld;
                    std::vector<int32_t> pkeys;   // distinct x of P in order, and their row positions
                    std::vector<int32_t> prow;
                    std::vector<Ent> ein, eout;
                    for (auto& pe : P) {
                        if (pkeys.empty() || pkeys.back() != pe.second.x) { pkeys.push_back(pe.second.x); prow.push_back(pe.first); }
                        ein.push_back(Ent{pe.second.y, (int)pkeys.size() - 1, pe.second.src});
                    }
                    std::map<long long, int> pcol;
                    for (auto& qe : Q) {
                        pcol[qe.second.x] = qe.first;
                        eout.push_back(Ent{qe.second.x, qe.second.y, qe.second.src});
                    }
                    dn.nP = (int)pkeys.size();
                    ib_build(ein, ident, dn.in);
                    ib_build(eout, [&](long long x) { return (long long)pcol[x]; }, dn.out);
                    dn.cmoff = (long long)ibmap.size();
                    ibmap.insert(ibmap.end(), prow.begin(), prow.end());
                    ib_maxP = std::max(ib_maxP, dn.nP);
                    ib_dense[B.root_level].push_back(dn);
                };
                for (int j : tj) {
                    const NodeRT& n = nd[j];
                    auto rc = in_range(B, n.c0, n.c0 + n.c);
                    if (rc.first == rc.second) continue;
                    if (!n.compressed) {   // an uncompressed panel outside every block: rows C_j and R_j
                        const int32_t* Rj = S.R(j);
                        std::vector<std::pair<int, IbEntry>> P, Q;
                        for (auto it = rc.first; it != rc.second; ++it) {
                            P.push_back({(int)(it->x - n.c0), *it});
                            Q.push_back({(int)(it->x - n.c0), *it});
                        }
                        for (auto it = rc.second; it != B.adj.end(); ++it) {
                            const int pos = (int)(std::lower_bound(Rj, Rj + n.r, it->x) - Rj);
                            if (pos < n.r && Rj[pos] == it->x) P.push_back({n.c + pos, *it});
                        }
                        region(P, Q, arena + n.off, n.ld);
                    } else if (!n.hier) {
                        std::vector<std::pair<int, IbEntry>> P;
                        for (auto it = rc.first; it != rc.second; ++it) P.push_back({(int)(it->x - n.c0), *it});
                        region(P, P, arena + n.off, n.c);
                    } else {
                        const BlockTree& bt = S.tree[j];
                        for (int sl = 1; sl <= bt.nblocks; ++sl) {
                            if (!bt.leaf[sl]) continue;
                            auto lr = in_range(B, n.c0 + bt.lo[sl], n.c0 + bt.hi[sl]);
                            std::vector<std::pair<int, IbEntry>> P;
                            for (auto it = lr.first; it != lr.second; ++it) P.push_back({(int)(it->x - n.c0 - bt.lo[sl]), *it});
                            region(P, P, arena + n.leaf_off[sl], bt.hi[sl] - bt.lo[sl]);
                        }
                    }
                }
            }
        }
        int32_t* d_sprp = pmem.upload(sp_rp, stream);
        int32_t* d_spci = pmem.upload(sp_ci, stream);
        d_spval = (double*)pmem.alloc(sizeof(double) * std::max<size_t>(sp_src.size(), 1));
        d_spsrc = pmem.upload(sp_src, stream);   // for values given on the device
        if (ib_on) {
            int32_t* d_ibmap = pmem.upload(ibmap, stream);
            auto resolve = [&](IbCsr& c) {
                if (c.pend < 0) return;
                const PendingBlk& pb = pend[c.pend];
                c.blk = CsrBlock{d_sprp + pb.rp_off, d_spci + pb.ci_off, d_spval + pb.v_off, pb.nrows, 0};
                c.rmap = d_ibmap + c.moff;
            };
            for (IBlock& B : iblocks) { resolve(B.fwd); resolve(B.bwd); }
            for (NodeRT& n : nd)
                for (auto& v : n.ibt)
                    for (IbTerm& t : v) { resolve(t.in_f); resolve(t.out_f); resolve(t.in_t); resolve(t.out_t); }
            for (auto& v : ib_dense)
                for (IbDense& d : v) { resolve(d.in); resolve(d.out); d.cmap = d_ibmap + d.cmoff; }
            if (ib_maxP > 0) {
                std::vector<T> win((size_t)(2 * ib_maxP + 64) * 64, T(0));
                for (int i = 0; i < 64; ++i) win[(size_t)(ib_maxP + i) * 64 + i] = T(1);
                ib_win = pmem.upload(win, stream);
            }
            d_zero = (T*)pmem.alloc(256);
            CK(cudaMemsetAsync(d_zero, 0, 256, stream));
        }
        for (auto& pb : pend) {
            if (pb.node < 0) continue;   // interior-block factors, resolved above
            CsrBlock b{d_sprp + pb.rp_off, d_spci + pb.ci_off, d_spval + pb.v_off, pb.nrows, 0};
            NodeRT& n = nd[pb.node];
            if (pb.label == 0) (pb.orient == 0 ? n.aR : n.aC) = b;
            else (pb.orient == 0 ? n.bR[pb.label] : n.bC[pb.label]) = b;
        }

        // tail maps for compressed nodes: positions of R_k[p1..] inside R_j
        {
            std::vector<int32_t> tails;
            std::vector<std::pair<int, long long>> where;
            for (int j = 0; j < M; ++j) {
                NodeRT& n = nd[j];
                if (!n.compressed) continue;
                const int32_t* Rj = S.R(j);
                n.tail_off.clear();
                for (long long d = S.desc_ptr[j]; d < S.desc_ptr[j + 1]; ++d) {
                    const int k = S.desc_k[d];
                    const int32_t* Rk = S.R(k);
                    n.tail_off.push_back((long long)tails.size());
                    for (int p = S.desc_p1[d]; p < S.nrows(k); ++p)
                        tails.push_back((int32_t)(std::lower_bound(Rj, Rj + n.r, Rk[p]) - Rj));
                }
            }
            int32_t* d_tails = pmem.upload(tails, stream);
            for (int j = 0; j < M; ++j)
                if (nd[j].compressed) nd[j].tailpos = d_tails;
        }

        // panel factorization steps per level (uncompressed panels and dense diagonals)
        panel_steps.assign(S.nlevels, {});
        for (int l = 0; l < S.nlevels; ++l) {
            std::vector<int> pan;
            for (int j : S.level_nodes[l])
                if (!nd[j].compressed || !nd[j].hier) pan.push_back(j);
            int maxc = 0;
            for (int j : pan) maxc = std::max(maxc, nd[j].c);
            for (int t0 = 0; t0 < maxc; t0 += NB) {
                std::vector<PotrfTask> pt;
                std::vector<TrsmTask> tt;
                std::vector<GemmTask> gt;
                for (int j : pan) {
                    const NodeRT& n = nd[j];
                    if (t0 >= n.c) continue;
                    const int nrows_tot = n.compressed ? n.c : n.c + n.r;
                    append_panel_step(arena + n.off, n.ld, n.c, nrows_tot, t0, j, pt, tt, gt);
                }
                double fp = 0, ft = 0, fg = 0;
                for (auto& x : pt) fp += (double)x.nb * x.nb * x.nb / 3.0;
                for (auto& x : tt) ft += (double)x.nrows * x.nb * x.nb;
                for (auto& x : gt) fg += x.lower ? (double)x.m * (x.n + 1) * x.K : 2.0 * x.m * x.n * x.K;
                PanelStep ps{pmem.upload(pt, stream), (int)pt.size(), pmem.upload(tt, stream), (int)tt.size(),
                             pmem.upload(gt, stream), (int)gt.size(), fp, ft, fg};
                panel_steps[l].push_back(ps);
            }
        }

        // inverses of the dense diagonal blocks factored by the level's panel steps
        inv_tasks.assign(S.nlevels, nullptr);
        inv_count.assign(S.nlevels, 0);
        inv_maxc.assign(S.nlevels, 0);
        for (int l = 0; l < S.nlevels; ++l) {
            std::vector<TrsvTask> tv;
            for (int j : S.level_nodes[l])
                if (!nd[j].hier) {
                    auto v = inverse_tasks_dense(j);
                    tv.insert(tv.end(), v.begin(), v.end());
                }
            for (auto& t : tv) inv_maxc[l] = std::max(inv_maxc[l], t.c);
            inv_tasks[l] = pmem.upload(tv, stream);
            inv_count[l] = (int)tv.size();
        }
        // push tasks per level: sources k of the level, every ancestor run, 64x64 tiles
        push_tasks.assign(S.nlevels, nullptr);
        push_count.assign(S.nlevels, 0);
        {
            std::vector<std::vector<PushTask>> byl(S.nlevels);
            std::vector<double> elems(M, 0.0), prow(M, 0.0);
            for (int j = 0; j < M; ++j)
                for (long long d = S.desc_ptr[j]; d < S.desc_ptr[j + 1]; ++d) {
                    const int k = S.desc_k[d];
                    if (nd[k].ib >= 0 && nd[j].ib != nd[k].ib) continue;   // Section 5.1: the closed forms
                    const int p0 = S.desc_p0[d], p1 = S.desc_p1[d], rk = nd[k].r;
                    const int rend = nd[j].compressed ? p1 : rk;
                    const double w = p1 - p0, h = rend - p0;
                    elems[k] += w * (w + 1) / 2 + (h - w) * w;
                    prow[k] += h;
                    for (int pc = p0; pc < p1; pc += TILE)
                        for (int pr = pc; pr < rend; pr += TILE)
                            byl[S.level[k]].push_back(
                                PushTask{k, j, pr, std::min(pr + TILE, rend), pc, std::min(pc + TILE, p1)});
                }
            push_elems.assign(S.nlevels, {});
            for (int k = 0; k < M; ++k)
                if (elems[k] > 0) push_elems[S.level[k]].push_back(PushElems{k, elems[k], prow[k]});
            for (int l = 0; l < S.nlevels; ++l) {
                push_tasks[l] = pmem.upload(byl[l], stream);
                push_count[l] = (int)byl[l].size();
            }
            push_tasks_tc.assign(S.nlevels, nullptr);
            push_count_tc.assign(S.nlevels, 0);
            if (tc) {
                std::vector<std::vector<PushTask>> bt(S.nlevels);
                for (int j = 0; j < M; ++j)
                    for (long long d = S.desc_ptr[j]; d < S.desc_ptr[j + 1]; ++d) {
                        const int k = S.desc_k[d];
                        if (nd[k].ib >= 0 && nd[j].ib != nd[k].ib) continue;
                        const int p0 = S.desc_p0[d], p1 = S.desc_p1[d], rk = nd[k].r;
                        const int rend = nd[j].compressed ? p1 : rk;
                        for (int pc = p0; pc < p1; pc += TC_N)
                            for (int pr = pc; pr < rend; pr += TC_M)
                                bt[S.level[k]].push_back(
                                    PushTask{k, j, pr, std::min(pr + TC_M, rend), pc, std::min(pc + TC_N, p1)});
                    }
                for (int l = 0; l < S.nlevels; ++l) {
                    push_tasks_tc[l] = pmem.upload(bt[l], stream);
                    push_count_tc[l] = (int)bt[l].size();
                }
            }
        }
        if (dense_graph) { cudaGraphExecDestroy(dense_graph); dense_graph = nullptr; }
        dense_prefix = 0;
        for (int l = 0; l < S.nlevels; ++l) {
            bool any = !ib_dense[l].empty();   // interior-block Schur complements run as programs
            for (int j : S.level_nodes[l]) any |= nd[j].compressed;
            if (any) break;
            dense_prefix = l + 1;
        }
        CK(cudaStreamSynchronize(stream));
        plan_compress = compress;
        plan_diag = diag;
        have_plan = true;
    }

    // one step of the blocked tall-panel Cholesky of panel P (nrows_tot x c, ld)
    static void append_panel_step(T* P, int ld, int c, int nrows_tot, int t0, int node, std::vector<PotrfTask>& pt,
                                  std::vector<TrsmTask>& tt, std::vector<GemmTask>& gt) {
        const int nb = std::min(NB, c - t0);
        T* D = P + t0 + (size_t)t0 * ld;
        pt.push_back(PotrfTask{D, ld, nb, node});
        for (int r0 = t0 + nb; r0 < nrows_tot; r0 += TILE)
            tt.push_back(TrsmTask{D, P + r0 + (size_t)t0 * ld, ld, ld, nb, std::min(TILE, nrows_tot - r0)});
        for (int c0 = t0 + nb; c0 < c; c0 += TILE) {
            const int ncol = std::min(TILE, c - c0);
            for (int r0 = c0; r0 < nrows_tot; r0 += TILE) {
                GemmTask g{};
                g.A = P + r0 + (size_t)t0 * ld;
                g.B = P + c0 + (size_t)t0 * ld;
                g.C = P + r0 + (size_t)c0 * ld;
                g.lda = ld; g.ldb = ld; g.ldc = ld;
                g.m = std::min(TILE, nrows_tot - r0);
                g.n = ncol;
                g.K = nb;
                g.moff = r0 - c0;
                g.lower = (r0 < c0 + ncol) ? 1 : 0;
                gt.push_back(g);
            }
        }
    }

    // ---------------------------------------------------------------- launch helpers
    void run_panel_steps(const std::vector<PanelStep>& steps) {
        for (const PanelStep& ps : steps) {
            if (ps.npotrf) { PROF(prof, "potrf", stream, ps.fl_potrf, 0, k_potrf_tile<T><<<ps.npotrf, 256, 0, stream>>>(ps.potrf, d_status)); launches++; }
            if (ps.ntrsm) { PROF(prof, "trsm", stream, ps.fl_trsm, 0, k_trsm_tile<T><<<ps.ntrsm, 256, 0, stream>>>(ps.trsm)); launches++; }
            if (ps.ngemm) { PROF(prof, "panel_gemm", stream, ps.fl_gemm, 0, k_gemm_tile<T><<<ps.ngemm, 256, 0, stream>>>(ps.gemm)); launches++; }
            LAUNCH_CHECK();
        }
    }

    // factor a batch of dense panels (nrows_tot x c each) together, step by step
    struct DensePanel { T* P; int ld; int c; int nrows_tot; int node; };
    void factor_dense_batch(const std::vector<DensePanel>& ps) {
        int maxc = 0;
        for (auto& d : ps) maxc = std::max(maxc, d.c);
        for (int t0 = 0; t0 < maxc; t0 += NB) {
            std::vector<PotrfTask> pt;
            std::vector<TrsmTask> tt;
            std::vector<GemmTask> gt;
            double fp = 0, ft = 0, fg = 0;
            for (auto& d : ps) {
                if (t0 >= d.c) continue;
                append_panel_step(d.P, d.ld, d.c, d.nrows_tot, t0, d.node, pt, tt, gt);
                flops += nb_flops(d.c, d.nrows_tot, t0);
            }
            for (auto& x : pt) fp += (double)x.nb * x.nb * x.nb / 3.0;
            for (auto& x : tt) ft += (double)x.nrows * x.nb * x.nb;
            for (auto& x : gt) fg += x.lower ? (double)x.m * (x.n + 1) * x.K : 2.0 * x.m * x.n * x.K;
            PotrfTask* dp = (PotrfTask*)upload_tmp(sTask, pt);
            PROF(prof, "potrf", stream, fp, 0, k_potrf_tile<T><<<(int)pt.size(), 256, 0, stream>>>(dp, d_status));
            launches++;
            if (!tt.empty()) {
                TrsmTask* dt = (TrsmTask*)upload_tmp(sTask2, tt);
                PROF(prof, "trsm", stream, ft, 0, k_trsm_tile<T><<<(int)tt.size(), 256, 0, stream>>>(dt));
                launches++;
            }
            if (!gt.empty()) {
                GemmTask* dg = (GemmTask*)upload_tmp(sT2, gt);
                PROF(prof, "panel_gemm", stream, fg, 0, k_gemm_tile<T><<<(int)gt.size(), 256, 0, stream>>>(dg));
                launches++;
            }
            LAUNCH_CHECK();
        }
    }
    static double nb_flops(int c, int nrows_tot, int t0) {
        const double nb = std::min(NB, c - t0);
        const double below = nrows_tot - t0 - nb;
        const double trail = c - t0 - nb;
        return nb * nb * nb / 3.0 + below * nb * nb + 2.0 * nb * (trail * (below - trail) + trail * (trail + 1) / 2.0);
    }

    // Task records go to a bump-allocated device arena; it is reset only when the
    // stream is idle (sync_stream), so records of kernels in flight stay valid.
    // cudaMemcpyAsync from pageable memory stages the data before returning.
    char* arena_base = nullptr;
    char* arena_host = nullptr;     // pinned staging mirror of the device arena
    size_t arena_cap = 0, arena_used = 0;
    void sync_stream() {
        if (prof.on) {
            const double t0 = now_ms();
            CK(cudaStreamSynchronize(stream));
            prof.wall("host_sync_wait", now_ms() - t0);
        } else {
            CK(cudaStreamSynchronize(stream));
        }
        arena_used = 0;
    }
    struct HostTimer {           // host time of a region, profile mode only
        EngineT* e; const char* name; double t0;
        HostTimer(EngineT* e_, const char* n) : e(e_), name(n), t0(e_->prof.on ? now_ms() : 0.0) {}
        ~HostTimer() { if (e->prof.on) e->prof.wall(name, now_ms() - t0); }
    };
    static double now_ms() {
        return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
    }
    // One region of the arena: fill(host staging, device address) writes the records (which may
    // point into the region itself), then one copy is queued.  A wrap or a larger arena (after a
    // stream synchronisation) happens only here, before the region is handed out, so records a
    // later upload displaces were consumed by launches already queued -- provided every launch
    // takes its records from a single upload (a launch whose records span two uploads could find
    // the first one overwritten or freed by the second).
    template <class F> char* upload_fill(size_t nbytes, F&& fill) {
        HostTimer ht_(this, "h_upload");
        const size_t bytes = (std::max<size_t>(nbytes, 1) + 255) / 256 * 256;
        if (arena_used + bytes > arena_cap) {
            sync_stream();
            if (bytes > arena_cap) {
                if (arena_base) CK(cudaFree(arena_base));
                if (arena_host) CK(cudaFreeHost(arena_host));
                arena_cap = std::max(bytes, (size_t)64 << 20);
                CK(cudaMalloc(&arena_base, arena_cap));
                CK(cudaMallocHost(&arena_host, arena_cap));
            }
        }
        char* p = arena_base + arena_used;
        if (nbytes) {
            fill(arena_host + arena_used, p);
            CK(cudaMemcpyAsync(p, arena_host + arena_used, nbytes, cudaMemcpyHostToDevice, stream));
        }
        arena_used += bytes;
        return p;
    }
    template <class X> void* upload_tmp(Scratch&, const std::vector<X>& v) {
        return upload_fill(sizeof(X) * v.size(), [&](char* h, char*) { std::memcpy(h, v.data(), sizeof(X) * v.size()); });
    }

    // ---------------------------------------------------------------- stage programs
    // An operation of one supernode (an implicit product, a hierarchical solve, ...)
    // is a list of stages.  Stage i of every node in a batch is launched together,
    // phase A (copies, samples, sparse products, triangular solves) before phase B
    // (TN products) before phase C (NN products); a stage never holds two phase-A
    // records that touch the same buffer.
    struct Stage {
        std::vector<HAct> hacts;           // actions of the hsolve tasks (acts holds an index here)
        std::vector<HTask> hs;
        std::vector<GaussTask> gauss;
        std::vector<CopyTask> copy;
        std::vector<CsrTask> csr;
        std::vector<TrsvTask> trsv;
        std::vector<TnTask> tn;
        std::vector<NnTask> nn;
    };
    using Program = std::vector<Stage>;
    static constexpr int TRSV_CW = sizeof(T) == 8 ? 1 : 8;   // FP64: spread columns over more SMs

    static TnTask tn_task(const void* A, int lda, int K, int nrow, const int32_t* amap, int aoff, const int32_t* ymap,
                          int yoff, const void* Y, int ldy, void* Z, int ldz, int N, double alpha = 1.0,
                          double beta = 0.0) {
        TnTask t{};
        t.A = A; t.lda = lda; t.K = K; t.nrow = nrow; t.amap = amap; t.aoff = aoff; t.ymap = ymap; t.yoff = yoff;
        t.Z = Z; t.ldz = ldz; t.t0 = 0; t.Y = Y; t.ldy = ldy; t.N = N; t.alpha = alpha; t.beta = beta;
        return t;
    }
    static NnTask nn_task(const void* A, int lda, int K, int nrow, const int32_t* amap, int aoff, const int32_t* ymap,
                          int yoff, const void* Z, int ldz, void* Y, int ldy, int N, double alpha, bool atomic) {
        NnTask t{};
        t.A = A; t.lda = lda; t.K = K; t.nrow = nrow; t.amap = amap; t.aoff = aoff; t.ymap = ymap; t.yoff = yoff;
        t.Z = Z; t.ldz = ldz; t.row0 = 0; t.Y = Y; t.ldy = ldy; t.N = N; t.alpha = alpha; t.atomic = atomic ? 1 : 0;
        return t;
    }
    // columns of A per launched TN task: 128 for the tensor-core kernel, 64 for the SIMT one (the
    // stage keeps whole tasks; run() cuts them for the kernel variant it launches)
    int cur_tn_cols = TS_COLS;
    int tn_cols() const { return cur_tn_cols; }
    void add_tn(Stage& s, const TnTask& t) {
        if (t.K == 0 || t.nrow == 0 || t.N == 0) return;
        s.tn.push_back(t);
        flops += 2.0 * t.nrow * t.K * t.N;
    }
    void add_nn(Stage& s, const NnTask& t) {
        if (t.K == 0 || t.nrow == 0 || t.N == 0) return;
        for (int r0 = 0; r0 < t.nrow; r0 += NN_ROWS) { NnTask c = t; c.row0 = r0; s.nn.push_back(c); }
        flops += 2.0 * t.nrow * t.K * t.N;
    }
    void add_csr(Stage& s, const CsrBlock& b, const T* X, int ldx, T* Y, int ldy, int N) {
        for (int r0 = 0; r0 < b.nrows; r0 += 16) s.csr.push_back(CsrTask{b, X, ldx, Y, ldy, N, r0, 1.0});
    }
    static void add_copy(Stage& s, const T* src, long long ssr, long long ssc, T* dst, long long dsr, long long dsc, int m,
                         int nc) {
        if ((long long)m * nc > 0) s.copy.push_back(CopyTask{src, ssr, ssc, dst, dsr, dsc, m, nc});
    }
    void add_trsv(Stage& s, const T* L, int ld, int c, T* X, int ldx, int N, bool transpose) {
        if (c == 0 || N == 0) return;
        s.trsv.push_back(TrsvTask{L, ld, c, N, X, ldx, transpose ? 1 : 0});
        flops += (double)c * c * N;
    }
    static Stage& next(Program& P) { P.emplace_back(); return P.back(); }

    double task_flops(const TnTask& t) const { return 2.0 * t.nrow * std::min(tn_cols(), t.K - t.t0) * t.N; }
    static double task_flops(const NnTask& t) { return 2.0 * std::min(NN_ROWS, t.nrow - t.row0) * t.K * t.N; }
    static double task_flops(const TrsvTask& t) { return (double)t.c * t.c * t.N; }
    template <class X> static double task_flops(const X&) { return 0.0; }
    // algorithmic bytes of a TN product: A's rows once, Y's gathered rows once per task (counted
    // with its first 64-column tile), Z written once (and read when beta != 0)
    double task_bytes(const TnTask& t) const {
        const double cols = std::min(tn_cols(), t.K - t.t0);
        return sizeof(T) * (t.nrow * cols + (t.t0 == 0 ? t.nrow * (double)t.N : 0.0) +
                            cols * t.N * (t.beta != 0.0 ? 2.0 : 1.0));
    }
    static double task_bytes(const NnTask& t) {
        const double rows = std::min(NN_ROWS, t.nrow - t.row0);
        return sizeof(T) * (rows * t.K + 2.0 * rows * t.N + (double)t.K * t.N);
    }
    static double task_bytes(const TrsvTask& t) { return sizeof(T) * ((double)t.c * (t.c + 1) / 2 + 2.0 * t.c * t.N); }
    template <class X> static double task_bytes(const X&) { return 0.0; }
    template <class X, class F> void launch_kind(const char* name, std::vector<X>& all, int ychunks, F&& launch) {
        if (all.empty()) return;
        X* d = (X*)upload_tmp(sTask, all);
        double fl = 0, by = 0;
        if (prof.enabled(name))
            for (const X& t : all) { fl += task_flops(t); by += task_bytes(t); }
        PROF(prof, name, stream, fl, by, launch(d, (int)all.size(), ychunks));
        launches++;
        LAUNCH_CHECK();
    }

    // tensor-core thin products of the BF16 / TF32 forms (FP32 storage only)
    template <bool TF> static void tn_tc_np(const TnTask* d, dim3 g, int np, cudaStream_t s, int* err) {
        if (np == 16) k_tn_tc<TF, 16><<<g, 128, tp_smem_bytes<TF>(16), s>>>(d, err);
        else if (np == 32) k_tn_tc<TF, 32><<<g, 128, tp_smem_bytes<TF>(32), s>>>(d, err);
        else k_tn_tc<TF, 64><<<g, 128, tp_smem_bytes<TF>(64), s>>>(d, err);
    }
    template <bool TF> static void nn_tc_np(const NnTask* d, dim3 g, int np, cudaStream_t s, int* err) {
        if (np == 16) k_nn_tc<TF, 16><<<g, 128, tp_smem_bytes<TF>(16), s>>>(d, err);
        else if (np == 32) k_nn_tc<TF, 32><<<g, 128, tp_smem_bytes<TF>(32), s>>>(d, err);
        else k_nn_tc<TF, 64><<<g, 128, tp_smem_bytes<TF>(64), s>>>(d, err);
    }
    void launch_tn_tc(const TnTask* d, dim3 g, int np, cudaStream_t s) {
        if (tc_tf32) tn_tc_np<true>(d, g, np, s, d_status + 1);
        else tn_tc_np<false>(d, g, np, s, d_status + 1);
    }
    void launch_nn_tc(const NnTask* d, dim3 g, int np, cudaStream_t s) {
        if (tc_tf32) nn_tc_np<true>(d, g, np, s, d_status + 1);
        else nn_tc_np<false>(d, g, np, s, d_status + 1);
    }
    template <bool TF> static void tc_attrs() {
        for (int np : {16, 32, 64}) {
            const int b = tp_smem_bytes<TF>(np);
            if (np == 16) { CK(cudaFuncSetAttribute(k_tn_tc<TF, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, b));
                            CK(cudaFuncSetAttribute(k_nn_tc<TF, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, b)); }
            if (np == 32) { CK(cudaFuncSetAttribute(k_tn_tc<TF, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, b));
                            CK(cudaFuncSetAttribute(k_nn_tc<TF, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, b)); }
            if (np == 64) { CK(cudaFuncSetAttribute(k_tn_tc<TF, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize, b));
                            CK(cudaFuncSetAttribute(k_nn_tc<TF, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize, b)); }
        }
    }

    void run(std::vector<Program>& progs) {
        HostTimer ht_(this, "h_run");
        size_t len = 0;
        for (auto& p : progs) len = std::max(len, p.size());
        for (size_t i = 0; i < len; ++i) {
            Stage st;
            int yn_nn = 1, yn_csr = 1, yn_tr = 1;
            for (auto& p : progs) {
                if (i >= p.size()) continue;
                Stage& s = p[i];
                const long long hb = (long long)st.hacts.size();
                st.hacts.insert(st.hacts.end(), s.hacts.begin(), s.hacts.end());
                for (HTask h : s.hs) { h.acts = (const HAct*)(intptr_t)((intptr_t)h.acts + hb); st.hs.push_back(h); }
                st.gauss.insert(st.gauss.end(), s.gauss.begin(), s.gauss.end());
                st.copy.insert(st.copy.end(), s.copy.begin(), s.copy.end());
                st.csr.insert(st.csr.end(), s.csr.begin(), s.csr.end());
                st.trsv.insert(st.trsv.end(), s.trsv.begin(), s.trsv.end());
                st.tn.insert(st.tn.end(), s.tn.begin(), s.tn.end());
                st.nn.insert(st.nn.end(), s.nn.begin(), s.nn.end());
            }
            int np_nn = 16;
            double fl_nn = 0;
            for (auto& t : st.nn) {
                np_nn = std::max(np_nn, std::min(t.N, 64) <= 16 ? 16 : std::min(t.N, 64) <= 32 ? 32 : 64);
                fl_nn += 2.0 * std::min(NN_ROWS, t.nrow - t.row0) * (double)t.K * t.N;
            }
            // kernel variants of the thin products (BF16 / TF32 forms: SIMT or tensor cores), chosen
            // per (class, sample-column width, size) by the tuner
            const std::string knn = Tuner::key("nn", np_nn, fl_nn);
            const int vnn = (tc && !st.nn.empty()) ? tuner.pick(knn, 1) : 0;
            for (auto& t : st.nn) yn_nn = std::max(yn_nn, cdiv(t.N, vnn ? 64 : 16));
            for (auto& t : st.csr) yn_csr = std::max(yn_csr, cdiv(t.N, 16));
            for (auto& t : st.trsv) yn_tr = std::max(yn_tr, cdiv(t.N, TRSV_CW));
            const unsigned long long seed = o.seed;
            cudaStream_t s = stream;
            if (!st.hs.empty()) run_hsolve(st.hacts, st.hs, s);
            launch_kind("gauss", st.gauss, 1, [&](GaussTask* d, int n, int) { k_gauss<T><<<n, 256, 0, s>>>(d, seed); });
            launch_kind("copy", st.copy, 1, [&](CopyTask* d, int n, int) { k_copy<T><<<dim3(n, 32), 256, 0, s>>>(d); });
            launch_kind("csr", st.csr, yn_csr, [&](CsrTask* d, int n, int y) { k_csr_mm<T><<<dim3(n, y), 256, 0, s>>>(d); });
            int maxn_tr = 0;
            for (auto& t : st.trsv) maxn_tr = std::max(maxn_tr, t.N);
            if (maxn_tr >= 32)   // many right-hand sides: the tiled form
                launch_kind("trsv", st.trsv, cdiv(maxn_tr, TT_COLS), [&](TrsvTask* d, int n, int y) {
                    k_trsv_tile<T><<<dim3(n, y), 256, tt_smem_bytes<T>(), s>>>(d);
                });
            else
                launch_kind("trsv", st.trsv, yn_tr,
                            [&](TrsvTask* d, int n, int y) { k_trsv<T, TRSV_CW><<<dim3(n, y), 256, 0, s>>>(d); });
            int zs_tn = 1, yc_tn = 1, np_tn = 16;
            double fl_tn = 0;
            for (auto& t : st.tn) {
                np_tn = std::max(np_tn, std::min(t.N, 64) <= 16 ? 16 : std::min(t.N, 64) <= 32 ? 32 : 64);
                fl_tn += 2.0 * t.nrow * (double)t.K * t.N;
            }
            const std::string ktn = Tuner::key("tn", np_tn, fl_tn);
            const int vtn = (tc && !st.tn.empty()) ? tuner.pick(ktn, 0) : 0;
            cur_tn_cols = vtn ? TP_M : TS_COLS;
            {   // whole tasks -> column tiles of the chosen kernel
                std::vector<TnTask> cut;
                cut.reserve(st.tn.size() * 2);
                for (const TnTask& t : st.tn)
                    for (int t0 = 0; t0 < t.K; t0 += cur_tn_cols) { TnTask c = t; c.t0 = t0; cut.push_back(c); }
                st.tn.swap(cut);
            }
            {   // long row ranges: split the rows over CTAs (deterministic fixed-order reduction)
                int coff = 0;
                for (auto& t : st.tn) {
                    const int ych = cdiv(t.N, 64);
                    yc_tn = std::max(yc_tn, ych);
                    if (t.nrow < TN_SPLIT_MIN || coff + ych > TN_CNT_CAP) continue;
                    t.nsplit = std::min(cdiv(t.nrow, TN_SPLIT_ROWS), TN_SPLIT_MAX);
                    t.rps = cdiv(t.nrow, t.nsplit);
                    t.part = wsT((size_t)t.nsplit * tn_cols() * t.N);
                    t.cnt = d_tncnt + coff;
                    coff += ych;
                    zs_tn = std::max(zs_tn, t.nsplit);
                }
            }
            launch_kind(vtn ? "tn_tc" : "tn", st.tn, yc_tn, [&](TnTask* d, int n, int y) {
                const dim3 g((unsigned)n, (unsigned)y, (unsigned)zs_tn);
                Tuner::Timed tt(tuner, tc ? ktn : std::string(), vtn, fl_tn, s);
                if (vtn) launch_tn_tc(d, g, np_tn, s);
                else if (np_tn == 16) k_tn_s<T, 16><<<g, 256, ts_smem_bytes<T>(16), s>>>(d);
                else if (np_tn == 32) k_tn_s<T, 32><<<g, 256, ts_smem_bytes<T>(32), s>>>(d);
                else k_tn_s<T, 64><<<g, 256, ts_smem_bytes<T>(64), s>>>(d);
            });
            launch_kind(vnn ? "nn_tc" : "nn", st.nn, yn_nn, [&](NnTask* d, int n, int y) {
                Tuner::Timed tt(tuner, tc ? knn : std::string(), vnn, fl_nn, s);
                if (vnn) launch_nn_tc(d, dim3((unsigned)n, (unsigned)y), np_nn, s);
                else k_nn<T><<<dim3(n, y), NN_ROWS, 0, s>>>(d);
            });
        }
        progs.clear();
    }

    // ---------------------------------------------------------------- per-batch device workspace
    // chunked bump allocator; reset() recycles every chunk (call with the stream idle)
    struct Workspace {
        std::vector<std::pair<char*, size_t>> chunks;
        size_t cur = 0, used = 0;
        ~Workspace() { for (auto& c : chunks) cudaFree(c.first); }
        void reset() { cur = 0; used = 0; }
        void* getb(size_t nbytes) {
            size_t bytes = (std::max<size_t>(nbytes, 1) + 255) / 256 * 256;
            while (true) {
                if (cur < chunks.size() && used + bytes <= chunks[cur].second) {
                    char* p = chunks[cur].first + used;
                    used += bytes;
                    return p;
                }
                if (cur + 1 < chunks.size() || (cur < chunks.size() && used > 0)) {
                    if (cur + 1 < chunks.size()) { ++cur; used = 0; continue; }
                }
                size_t sz = std::max(bytes, (size_t)256 << 20);
                char* p = nullptr;
                CK(cudaMalloc(&p, sz));
                chunks.emplace_back(p, sz);
                cur = chunks.size() - 1;
                used = 0;
            }
        }
    };
    Workspace ws;
    T* wsT(size_t n) { return (T*)ws.getb(sizeof(T) * n); }
    // t buffers of the interior-block terms, kept for the products that write the same output
    // (the passes of one range finder reuse theirs; the workspace reset drops them)
    std::map<std::tuple<const void*, int, int, int>, T*> ib_tcache;
    void ws_reset() { ws.reset(); ib_tcache.clear(); }

    // ---------------------------------------------------------------- interior blocks (programs)
    // Stage i of sub joins stage at + i of P.
    static void merge_into(Program& P, size_t at, Program& sub) {
        if (P.size() < at + sub.size()) P.resize(at + sub.size());
        for (size_t i = 0; i < sub.size(); ++i) {
            Stage& d = P[at + i];
            Stage& s = sub[i];
            const long long hb = (long long)d.hacts.size();
            d.hacts.insert(d.hacts.end(), s.hacts.begin(), s.hacts.end());
            for (HTask h : s.hs) { h.acts = (const HAct*)(intptr_t)((intptr_t)h.acts + hb); d.hs.push_back(h); }
            d.gauss.insert(d.gauss.end(), s.gauss.begin(), s.gauss.end());
            d.copy.insert(d.copy.end(), s.copy.begin(), s.copy.end());
            d.csr.insert(d.csr.end(), s.csr.begin(), s.csr.end());
            d.trsv.insert(d.trsv.end(), s.trsv.begin(), s.trsv.end());
            d.tn.insert(d.tn.end(), s.tn.begin(), s.tn.end());
            d.nn.insert(d.nn.end(), s.nn.begin(), s.nn.end());
        }
    }
    static void add_csr_map(Stage& s, const IbCsr& b, const T* X, int ldx, T* Y, int ldy, int N, double alpha,
                            const int32_t* cmap, int mode, int lower) {
        for (int r0 = 0; r0 < b.blk.nrows; r0 += 16) {
            CsrTask t{b.blk, X, ldx, Y, ldy, N, r0, alpha};
            t.rmap = b.rmap;
            t.cmap = cmap;
            t.mode = mode;
            t.lower = lower;
            s.csr.push_back(t);
        }
    }
    // t (|C_B| x N, row-major, rows local to C_B) <- L_B^{-1} t or L_B^{-T} t: the block's
    // supernodes level by level, each with its diagonal solve and its panel rows inside C_B.
    void prog_block_solve(Program& P, int b, T* t, int N, bool transpose) {
        const IBlock& B = iblocks[b];
        const int nl = (int)B.lvl.size();
        for (int li = 0; li < nl; ++li) {
            const int lv = transpose ? nl - 1 - li : li;
            const std::vector<int>& nodes = B.lvl[lv];
            if (nodes.empty()) continue;
            if (transpose) {   // t[C_k] -= L(R_k in C_B, C_k)^T t[R_k in C_B]
                Stage st;
                for (int k : nodes) {
                    const NodeRT& n = nd[k];
                    add_tn(st, tn_task(arena + n.off + n.c, n.ld, n.c, n.r, nullptr, 0, d_rows + S.rows_ptr[k], (int)-B.c0,
                                       t, N, t + (size_t)(n.c0 - B.c0) * N, N, N, -1.0, 1.0));
                }
                if (!st.tn.empty()) P.push_back(std::move(st));
            }
            const size_t base = P.size();
            for (int k : nodes) {
                Program sub;
                prog_diag_solve(sub, k, 0, t + (size_t)(nd[k].c0 - B.c0) * N, N, N, transpose);
                merge_into(P, base, sub);
            }
            if (!transpose) {   // t[R_k in C_B] -= L(R_k in C_B, C_k) t[C_k]; after the level's solves
                Stage& st = P.back();
                for (int k : nodes) {
                    const NodeRT& n = nd[k];
                    add_nn(st, nn_task(arena + n.off + n.c, n.ld, n.c, n.r, nullptr, 0, d_rows + S.rows_ptr[k], (int)-B.c0,
                                       t + (size_t)(n.c0 - B.c0) * N, N, t, N, N, -1.0, true));
                }
            }
        }
    }
    // Eq. interiorBlockMult for every interior block meeting label s of supernode j: stage `at` of
    // P starts W(out) -= A(out, C_B) L_B^{-T} L_B^{-1} A(C_B, in) X (in / out: columns / rows of the
    // block of L, exchanged for the transpose); the terms end before the stages appended after.
    void ib_chains(Program& P, size_t at, int j, int s, bool transpose, const T* X, int ldx, T* W, int ldw, int N) {
        const NodeRT& n = nd[j];
        if ((int)n.ibt.size() <= s) return;
        for (size_t i = 0; i < n.ibt[s].size(); ++i) {
            const IbTerm& tm = n.ibt[s][i];
            const IBlock& B = iblocks[tm.b];
            const IbCsr& in = transpose ? tm.in_t : tm.in_f;
            const IbCsr& out = transpose ? tm.out_t : tm.out_f;
            const int nb = (int)(B.c1 - B.c0);
            T*& t = ib_tcache[std::make_tuple((const void*)W, s, (int)i, N)];
            if (!t) t = wsT((size_t)nb * N);
            Program sub;
            add_copy(next(sub), d_zero, 0, 0, t, 1, 0, nb * N, 1);   // t = 0 (contiguous), then the listed rows
            add_csr_map(sub.back(), in, X, ldx, t, N, N, 1.0, nullptr, 0, 0);
            prog_block_solve(sub, tm.b, t, N, false);
            prog_block_solve(sub, tm.b, t, N, true);
            add_csr_map(next(sub), out, t, N, W, ldw, N, -1.0, nullptr, 2, 0);
            merge_into(P, at, sub);
        }
    }
    // Schur complements of the blocks whose root is at level l into their dense targets,
    // C(P, Q) = A(P, C_B) L_B^{-T} L_B^{-1} A(C_B, Q) for 64 columns of P per program, the
    // lower triangle subtracted in place (Section 5.1: the needed sub-blocks of L(R_B, C_B)
    // appear only through the closed form).
    static constexpr size_t IB_WS_CAP = (size_t)512 << 20;
    void ib_dense_level(int l) {
        if (!ib_on || ib_dense[l].empty()) return;
        const std::string keep_tag = prof.tag;
        prof.tag += "@ibd";
        const std::vector<IbDense>& v = ib_dense[l];
        size_t i = 0;
        while (i < v.size()) {
            ws_reset();
            std::vector<Program> progs;
            size_t bytes = 0;
            for (; i < v.size() && bytes < IB_WS_CAP; ++i) {
                const IbDense& d = v[i];
                const IBlock& B = iblocks[d.b];
                const int nb = (int)(B.c1 - B.c0);
                for (int p0 = 0; p0 < d.nP; p0 += 64) {
                    const int N = std::min(64, d.nP - p0);
                    T* t = wsT((size_t)nb * N);
                    bytes += sizeof(T) * (size_t)nb * N;
                    progs.emplace_back();
                    Program& P = progs.back();
                    add_copy(next(P), d_zero, 0, 0, t, 1, 0, nb * N, 1);
                    // columns p0 .. p0 + N - 1 of the identity over P: the window's rows ib_maxP ..
                    add_csr_map(P.back(), d.in, ib_win + (size_t)(ib_maxP - p0) * 64, 64, t, N, N, 1.0, nullptr, 0, 0);
                    prog_block_solve(P, d.b, t, N, false);
                    prog_block_solve(P, d.b, t, N, true);
                    add_csr_map(next(P), d.out, t, N, d.base, d.ld, N, -1.0, d.cmap + p0, 2, 1);
                }
            }
            run(progs);
        }
        prof.tag = keep_tag;
    }

    // ---------------------------------------------------------------- dense / hierarchical triangular solves (programs)
    // Action list of the solve with the subtree of L^D_j rooted at s (0: whole block),
    // rows relative to the subtree's first row (Alg. 4, branches in the corrected order).
    void hacts(int j, int s, bool transpose, std::vector<HAct>& out) {
        const NodeRT& n = nd[j];
        if (!n.hier) {
            const T* L = arena + n.off;
            const int ld = n.ld, c = n.c, bs = SOLVE_MAX, nblk = cdiv(c, bs);
            for (int bi = 0; bi < nblk; ++bi) {
                const int b = transpose ? nblk - 1 - bi : bi;
                const int b0 = b * bs, b1 = std::min(c, b0 + bs);
                out.push_back(HAct{HA_TRSV, 0, 0, b0, b1 - b0, 0, inv_block(j, b0), b1 - b0, nullptr, 0});
                if (!transpose && b1 < c)
                    out.push_back(HAct{HA_GEMV, b0, 0, b1, c - b1, b1 - b0, nullptr, 0, L + b1 + (size_t)b0 * ld, ld});
                if (transpose && b0 > 0)
                    out.push_back(HAct{HA_GEMVT, b0, b1 - b0, 0, b0, 0, L + b0, ld, nullptr, 0});
                flops += (double)(b1 - b0) * (b1 - b0) + 2.0 * (b1 - b0) * (transpose ? b0 : c - b1);
            }
            return;
        }
        const BlockTree& t = S.tree[j];
        if (s == 0) s = t.root;
        const int base = t.lo[s];
        std::function<void(int)> rec = [&](int b) {
            if (t.leaf[b]) {
                const int sz = t.hi[b] - t.lo[b];
                out.push_back(HAct{HA_TRSV, 0, 0, t.lo[b] - base, sz, 0, invs + n.leaf_inv[b], sz, nullptr, 0});
                flops += (double)sz * sz;
                return;
            }
            const int n1 = t.mid[b] - t.lo[b], n2 = t.hi[b] - t.mid[b], q = n.brank[b];
            auto lowrank = [&]() {
                if (!q) return;
                if (!transpose)
                    out.push_back(HAct{HA_LR, t.lo[b] - base, n1, t.mid[b] - base, n2, q, n.bU[b], n1, n.bV[b], n2});
                else
                    out.push_back(HAct{HA_LR, t.mid[b] - base, n2, t.lo[b] - base, n1, q, n.bV[b], n2, n.bU[b], n1});
                flops += 2.0 * q * (n1 + n2);
            };
            if (!transpose) { rec(t.left[b]); lowrank(); rec(t.right[b]); }
            else { rec(t.right[b]); lowrank(); rec(t.left[b]); }
        };
        rec(s);
    }
    // column chunk of the persistent solve so that (c + Z rows) x CW fits in shared memory
    static int pick_cw(int c) {
        const size_t cap = 200 * 1024;
        for (int cw : {8, 4, 2, 1})
            if ((size_t)(c + HS_ZROWS) * cw * sizeof(T) <= cap) return cw;
        return 0;
    }
    static size_t hs_smem(int c, int cw) { return (size_t)(c + HS_ZROWS) * cw * sizeof(T); }
    // dynamic shared memory of k_leaf_factor for an sz-column leaf (block + FP64 tile)
    static constexpr size_t LEAF_SMEM_CAP = 220 * 1024;
    static size_t leaf_smem(int sz) { return ((size_t)sizeof(T) * sz * leaf_ld(sz) + 15) / 16 * 16 + LP * LEAF_DT * 8; }
    template <int CW> static void hs_attr() {
        CK(cudaFuncSetAttribute(k_hsolve<T, CW>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024 + 256));
    }
    // launch persistent solves, one launch per column chunk width; tasks' acts are device pointers.
    // At most 4 columns per CTA: the hierarchical chain's solves have few tasks, and twice the
    // CTAs walking the action list beat the wider chunk (96^3: 14.2 -> 11.5 ms; 2 columns: 14.6)
    static constexpr int HS_CW_MAX = 4;
    void run_hsolve(const std::vector<HAct>& acts, const std::vector<HTask>& tasks, cudaStream_t s) {
        // tasks[i].acts holds an index into acts.  The actions and every width group's task list
        // go up in one upload: a second upload could wrap the arena over the first one before the
        // kernels that read both have run
        const int widths[4] = {8, 4, 2, 1};
        std::vector<HTask> grp[4];
        int maxc[4] = {0, 0, 0, 0}, ych[4] = {1, 1, 1, 1};
        for (const HTask& t : tasks) {
            const int w = std::min(pick_cw(t.c), HS_CW_MAX);
            const int g = w == 8 ? 0 : w == 4 ? 1 : w == 2 ? 2 : 3;
            grp[g].push_back(t);
            maxc[g] = std::max(maxc[g], t.c);
            ych[g] = std::max(ych[g], cdiv(t.N, w));
        }
        auto al = [](size_t x) { return (x + 255) / 256 * 256; };
        size_t off[4], total = al(sizeof(HAct) * acts.size());
        for (int g = 0; g < 4; ++g) { off[g] = total; total += al(sizeof(HTask) * grp[g].size()); }
        char* d = upload_fill(total, [&](char* h, char* dd) {
            if (!acts.empty()) std::memcpy(h, acts.data(), sizeof(HAct) * acts.size());
            for (int g = 0; g < 4; ++g)
                for (size_t i = 0; i < grp[g].size(); ++i) {
                    HTask t = grp[g][i];
                    t.acts = (const HAct*)dd + (intptr_t)t.acts;
                    std::memcpy(h + off[g] + sizeof(HTask) * i, &t, sizeof(HTask));
                }
        });
        for (int g = 0; g < 4; ++g) {
            if (grp[g].empty()) continue;
            const HTask* dt = (const HTask*)(d + off[g]);
            const dim3 grid((unsigned)grp[g].size(), (unsigned)ych[g]);
            const size_t sm = hs_smem(maxc[g], widths[g]);
            switch (widths[g]) {
                case 8: PROF(prof, "hsolve", s, 0, 0, k_hsolve<T, 8><<<grid, HS_THREADS, sm, s>>>(dt)); break;
                case 4: PROF(prof, "hsolve", s, 0, 0, k_hsolve<T, 4><<<grid, HS_THREADS, sm, s>>>(dt)); break;
                case 2: PROF(prof, "hsolve", s, 0, 0, k_hsolve<T, 2><<<grid, HS_THREADS, sm, s>>>(dt)); break;
                default: PROF(prof, "hsolve", s, 0, 0, k_hsolve<T, 1><<<grid, HS_THREADS, sm, s>>>(dt)); break;
            }
            launches++;
            LAUNCH_CHECK();
        }
    }
    // X (c x N row-major, ld ldx) <- L^{-1} X or L^{-T} X for dense lower L (ld), blocked by SOLVE_MAX
    void prog_dense_solve(Program& P, int j, T* X, int ldx, int N, bool transpose) {
        const NodeRT& n = nd[j];
        const T* L = arena + n.off;
        const int ld = n.ld, c = n.c;
        if (c == 0) return;
        const int bs = SOLVE_MAX, nblk = cdiv(c, bs);
        for (int bi = 0; bi < nblk; ++bi) {
            const int b = transpose ? nblk - 1 - bi : bi;
            const int b0 = b * bs, b1 = std::min(c, b0 + bs);
            Stage& s = next(P);
            add_trsv(s, inv_block(j, b0), b1 - b0, b1 - b0, X + (size_t)b0 * ldx, ldx, N, transpose);
            if (!transpose && b1 < c)
                add_nn(s, nn_task(L + b1 + (size_t)b0 * ld, ld, b1 - b0, c - b1, nullptr, 0, nullptr, 0, X + (size_t)b0 * ldx,
                                  ldx, X + (size_t)b1 * ldx, ldx, N, -1.0, false));
            if (transpose && b0 > 0)
                add_tn(s, tn_task(L + b0, ld, b0, b1 - b0, nullptr, 0, nullptr, 0, X + (size_t)b0 * ldx, ldx, X, ldx, N,
                                  -1.0, 1.0));
        }
    }

    // Alg. 4 (branches in the corrected order) on the subtree of L^D_j rooted at s (0 = root).
    void prog_diag_solve(Program& P, int j, int s, T* X, int ldx, int N, bool transpose) {
        const NodeRT& n = nd[j];
        if (!n.hier && n.c <= SOLVE_MAX) { prog_dense_solve(P, j, X, ldx, N, transpose); return; }
        const int c = n.hier ? (s == 0 ? n.c : S.tree[j].hi[s] - S.tree[j].lo[s]) : n.c;
        if (pick_cw(c) > 0) {
            Stage& st = next(P);
            const long long first = (long long)st.hacts.size();
            hacts(j, s, transpose, st.hacts);
            st.hs.push_back(HTask{(const HAct*)(intptr_t)first, (long long)st.hacts.size() - first, X, ldx, N, c,
                                  transpose ? 1 : 0});
            return;
        }
        if (!n.hier) { prog_dense_solve(P, j, X, ldx, N, transpose); return; }
        const BlockTree& t = S.tree[j];
        if (s == 0) s = t.root;
        if (t.leaf[s]) {
            const int sz = t.hi[s] - t.lo[s];
            add_trsv(next(P), invs + n.leaf_inv[s], sz, sz, X, ldx, N, transpose);
            return;
        }
        const int n1 = t.mid[s] - t.lo[s], n2 = t.hi[s] - t.mid[s], q = n.brank[s];
        T* X1 = X;
        T* X2 = X + (size_t)n1 * ldx;
        auto lowrank = [&]() {
            if (!q) return;
            T* Z = wsT((size_t)q * N);
            Stage& st = next(P);
            if (!transpose) {   // X2 -= V_s (U_s^T X1)
                add_tn(st, tn_task(n.bU[s], n1, q, n1, nullptr, 0, nullptr, 0, X1, ldx, Z, N, N));
                add_nn(st, nn_task(n.bV[s], n2, q, n2, nullptr, 0, nullptr, 0, Z, N, X2, ldx, N, -1.0, false));
            } else {            // X1 -= U_s (V_s^T X2)
                add_tn(st, tn_task(n.bV[s], n2, q, n2, nullptr, 0, nullptr, 0, X2, ldx, Z, N, N));
                add_nn(st, nn_task(n.bU[s], n1, q, n1, nullptr, 0, nullptr, 0, Z, N, X1, ldx, N, -1.0, false));
            }
        };
        if (!transpose) {
            prog_diag_solve(P, j, t.left[s], X1, ldx, N, false);
            lowrank();
            prog_diag_solve(P, j, t.right[s], X2, ldx, N, false);
        } else {
            prog_diag_solve(P, j, t.right[s], X2, ldx, N, true);
            lowrank();
            prog_diag_solve(P, j, t.left[s], X1, ldx, N, true);
        }
    }

    // ---------------------------------------------------------------- implicit products (programs)
    const LoOp& lo(int k) const { return h_lo[k]; }

    // Alg. 2 transposed: W (c x N) = (L^O_j)^T G, G (r x N); row-major, ld N.
    // X (c x N, row-major ld ldx) <- (L^D_j)^{-1} X or (L^D_j)^{-T} X for a hierarchical diagonal
    // block whose inverse factors tU_s, tV_s are formed: stage 1 the products with the input
    // (z_s = tU_s^T X[cols(s)], or tV_s^T X[rows(s)]), stage 2 the leaf inverses in place and
    // then X[rows(s)] -= tV_s z_s (or X[cols(s)] -= tU_s z_s), atomic over nested blocks.
    bool inverse_ready(int j) const {
        const NodeRT& n = nd[j];
        if (!n.hier) return false;
        const BlockTree& t = S.tree[j];
        for (int b = 1; b <= t.nblocks; ++b)
            if (!t.leaf[b] && n.brank[b] > 0 && !n.tU[b]) return false;
        return true;
    }
    void prog_diag_solve_inv(Program& P, int j, T* X, int ldx, int N, bool transpose) {
        const NodeRT& n = nd[j];
        const BlockTree& t = S.tree[j];
        std::vector<T*> zb(t.nblocks + 1, nullptr);
        Stage& st1 = next(P);
        for (int b = 1; b <= t.nblocks; ++b) {
            const int q = n.brank[b];
            if (t.leaf[b] || q == 0) continue;
            const int n1 = t.mid[b] - t.lo[b], n2 = t.hi[b] - t.mid[b];
            zb[b] = wsT((size_t)q * N);
            if (!transpose) add_tn(st1, tn_task(n.tU[b], n1, q, n1, nullptr, 0, nullptr, t.lo[b], X, ldx, zb[b], N, N));
            else add_tn(st1, tn_task(n.tV[b], n2, q, n2, nullptr, 0, nullptr, t.mid[b], X, ldx, zb[b], N, N));
        }
        Stage& st2 = next(P);
        for (int b = 1; b <= t.nblocks; ++b) {
            if (t.leaf[b]) {
                const int sz = t.hi[b] - t.lo[b];
                add_trsv(st2, invs + n.leaf_inv[b], sz, sz, X + (size_t)t.lo[b] * ldx, ldx, N, transpose);
                continue;
            }
            const int q = n.brank[b];
            if (q == 0) continue;
            const int n1 = t.mid[b] - t.lo[b], n2 = t.hi[b] - t.mid[b];
            if (!transpose) add_nn(st2, nn_task(n.tV[b], n2, q, n2, nullptr, 0, nullptr, t.mid[b], zb[b], N, X, ldx, N, -1.0, true));
            else add_nn(st2, nn_task(n.tU[b], n1, q, n1, nullptr, 0, nullptr, t.lo[b], zb[b], N, X, ldx, N, -1.0, true));
        }
    }

    void prog_offdiag_T(Program& P, int j, const T* G, int N, T* W) {
        const NodeRT& n = nd[j];
        const size_t base = P.size();
        Stage& st = next(P);
        add_csr(st, n.aC, G, N, W, N, N);
        int di = 0;
        for (long long d = S.desc_ptr[j]; d < S.desc_ptr[j + 1]; ++d, ++di) {
            const int k = S.desc_k[d];
            if (nd[k].ib >= 0) continue;   // interior blocks: the Eq. interiorBlockMult terms
            const LoOp& op = lo(k);
            const int p0 = S.desc_p0[d], p1 = S.desc_p1[d], rk = S.nrows(k);
            if (op.K == 0 || rk == p1) continue;          // empty R^O: no contribution
            T* Z = wsT((size_t)op.K * N);
            // T_k = L^O_k(R^O)^T gatherRows(G, R_j, R^O); W -= scatterRows(L^O_k(R^D) T_k, R^D, C_j)
            add_tn(st, tn_task(op.base, op.ld, op.K, rk - p1, nullptr, p1, n.tailpos + n.tail_off[di], 0, G, N, Z, N, N));
            add_nn(st, nn_task(op.base, op.ld, op.K, p1 - p0, nullptr, p0, d_rows + S.rows_ptr[k] + p0, (int)-n.c0, Z, N,
                               W, N, N, -1.0, true));
        }
        ib_chains(P, base, j, 0, true, G, N, W, N, N);
        if (inverse_ready(j)) prog_diag_solve_inv(P, j, W, N, N, false);
        else prog_diag_solve(P, j, 0, W, N, N, false);
    }

    // Alg. 2: W (r x N) = L^O_j X, X (c x N); Xp (c x N) is scratch.
    void prog_offdiag(Program& P, int j, const T* X, int N, T* W, T* Xp) {
        const NodeRT& n = nd[j];
        add_copy(next(P), X, N, 1, Xp, N, 1, n.c, N);
        if (inverse_ready(j)) prog_diag_solve_inv(P, j, Xp, N, N, true);
        else prog_diag_solve(P, j, 0, Xp, N, N, true);
        const size_t base = P.size();
        Stage& st = next(P);
        add_csr(st, n.aR, Xp, N, W, N, N);
        int di = 0;
        for (long long d = S.desc_ptr[j]; d < S.desc_ptr[j + 1]; ++d, ++di) {
            const int k = S.desc_k[d];
            if (nd[k].ib >= 0) continue;   // interior blocks: the Eq. interiorBlockMult terms
            const LoOp& op = lo(k);
            const int p0 = S.desc_p0[d], p1 = S.desc_p1[d], rk = S.nrows(k);
            if (op.K == 0 || rk == p1) continue;
            T* Z = wsT((size_t)op.K * N);
            // T_k = L^O_k(R^D)^T gatherRows(X', C_j, R^D); W -= scatterRows(L^O_k(R^O) T_k, R^O, R_j)
            add_tn(st, tn_task(op.base, op.ld, op.K, p1 - p0, nullptr, p0, d_rows + S.rows_ptr[k] + p0, (int)-n.c0, Xp, N,
                               Z, N, N));
            add_nn(st, nn_task(op.base, op.ld, op.K, rk - p1, nullptr, p1, n.tailpos + n.tail_off[di], 0, Z, N, W, N, N,
                               -1.0, true));
        }
        ib_chains(P, base, j, 0, false, Xp, N, W, N, N);
    }

    // positions of R_k inside the global range [g0, g1) (a sub-run of the C_j run)
    void run_in(long long d, long long g0, long long g1, int& a, int& b) const {
        const int k = S.desc_k[d];
        const int32_t* Rk = S.R(k);
        const int p0 = S.desc_p0[d], p1 = S.desc_p1[d];
        a = (int)(std::lower_bound(Rk + p0, Rk + p1, (int32_t)g0) - Rk);
        b = (int)(std::lower_bound(Rk + p0, Rk + p1, (int32_t)g1) - Rk);
    }

    // descendant and earlier-block terms of Alg. 5 (transpose = false) or its transpose
    void diag_terms(Stage& st, int j, int s, const T* In, int N, T* W, bool transpose) {
        const NodeRT& n = nd[j];
        const BlockTree& t = S.tree[j];
        const int r0 = t.mid[s], r1 = t.hi[s], q0 = t.lo[s], q1 = t.mid[s];
        // In has |cols| rows (Alg. 5) or |rows| rows (transpose); W the other
        const long long gin = n.c0 + (transpose ? r0 : q0), gout = n.c0 + (transpose ? q0 : r0);
        for (long long d = S.desc_ptr[j]; d < S.desc_ptr[j + 1]; ++d) {
            const int k = S.desc_k[d];
            if (nd[k].ib >= 0) continue;   // interior blocks: the Eq. interiorBlockMult terms
            const LoOp& op = lo(k);
            if (op.K == 0) continue;
            int a0, a1, b0, b1;
            run_in(d, n.c0 + r0, n.c0 + r1, a0, a1);    // rows of the block
            run_in(d, n.c0 + q0, n.c0 + q1, b0, b1);    // columns of the block
            if (a0 >= a1 || b0 >= b1) continue;
            const int i0 = transpose ? a0 : b0, i1 = transpose ? a1 : b1;
            const int o0 = transpose ? b0 : a0, o1 = transpose ? b1 : a1;
            T* Z = wsT((size_t)op.K * N);
            add_tn(st, tn_task(op.base, op.ld, op.K, i1 - i0, nullptr, i0, d_rows + S.rows_ptr[k] + i0, (int)-gin, In, N, Z,
                               N, N));
            add_nn(st, nn_task(op.base, op.ld, op.K, o1 - o0, nullptr, o0, d_rows + S.rows_ptr[k] + o0, (int)-gout, Z, N, W,
                               N, N, -1.0, true));
        }
        // earlier blocks p < s on the path to the root (U_p^T U_p = I)
        for (int p = t.parent[s]; p; p = t.parent[p]) {
            if (p > s || n.brank[p] == 0) continue;
            const int mp = t.hi[p] - t.mid[p], pr0 = t.mid[p];
            const int ioff = (transpose ? r0 : q0) - pr0, ooff = (transpose ? q0 : r0) - pr0;
            const int inr = transpose ? r1 - r0 : q1 - q0, outr = transpose ? q1 - q0 : r1 - r0;
            T* Z = wsT((size_t)n.brank[p] * N);
            add_tn(st, tn_task(n.bV[p], mp, n.brank[p], inr, nullptr, ioff, nullptr, 0, In, N, Z, N, N));
            add_nn(st, nn_task(n.bV[p], mp, n.brank[p], outr, nullptr, ooff, nullptr, 0, Z, N, W, N, N, -1.0, true));
        }
    }

    // Alg. 5: W (|rows_s| x N) = L^D_{j,s} X, X (|cols_s| x N); Xp scratch.
    void prog_diag_mult(Program& P, int j, int s, const T* X, int N, T* W, T* Xp) {
        const NodeRT& n = nd[j];
        const BlockTree& t = S.tree[j];
        const int cs = t.mid[s] - t.lo[s];
        add_copy(next(P), X, N, 1, Xp, N, 1, cs, N);
        prog_diag_solve(P, j, t.left[s], Xp, N, N, true);
        const size_t base = P.size();
        Stage& st = next(P);
        add_csr(st, n.bR[s], Xp, N, W, N, N);
        diag_terms(st, j, s, Xp, N, W, false);
        ib_chains(P, base, j, s, false, Xp, N, W, N, N);
    }

    // Alg. 5 transposed: W (|cols_s| x N) = (L^D_{j,s})^T G, G (|rows_s| x N).
    void prog_diag_mult_T(Program& P, int j, int s, const T* G, int N, T* W) {
        const NodeRT& n = nd[j];
        const BlockTree& t = S.tree[j];
        const size_t base = P.size();
        Stage& st = next(P);
        add_csr(st, n.bC[s], G, N, W, N, N);
        diag_terms(st, j, s, G, N, W, true);
        ib_chains(P, base, j, s, true, G, N, W, N, N);
        prog_diag_solve(P, j, t.left[s], W, N, N, false);
    }

    // ---------------------------------------------------------------- adaptive range finder (Alg. 3), batched
    T* lr_alloc(long long elems) {
        if (lr_used + elems > lr_cap) throw Error(RSC_ERR_OOM, "low-rank storage exhausted");
        T* p = lr_base + lr_used;
        lr_used += (elems + 31) / 32 * 32;
        return p;
    }

    struct RF {                    // one block being compressed
        int j = 0, s = 0;          // s == 0: L^O_j; else internal block s of L^D_j
        int m = 0, c = 0, maxr = 0;
        int cap = 1 << 30;         // largest rank: Eq. rankFunction in the fixed-rank form
        double tol = 0;
        uint32_t block_id = 0;
        T* U = nullptr; T* V = nullptr;
        int rank = 0;
        bool active = true;        // as last read back from the device
        T *Y = nullptr, *Gp = nullptr;
        T *Gb = nullptr, *Yb = nullptr;   // prefetched samples of PREFETCH passes (16 PREFETCH columns)
        int pref_base = 0, pref_n = 0;
        int passes = 0;
    };
    static constexpr int PREFETCH = 4;   // sampling passes whose products are formed together
    RfBarrier* d_rfbar = nullptr;
    RfDev<T>* rf_host = nullptr;         // pinned: upload of the batch records, read-back of their state
    size_t rf_host_cap = 0;
    int* st_host = nullptr;              // pinned: status words read back with the state
    int coop_max = 0;                    // co-resident CTAs of k_rf_pass
    unsigned long long* d_rfp_time = nullptr;   // profile mode: time per k_rf_pass phase (ns)

    void mult_T_prog(Program& P, RF& r, const T* G, int N, T* W) {
        if (r.s == 0) prog_offdiag_T(P, r.j, G, N, W);
        else prog_diag_mult_T(P, r.j, r.s, G, N, W);
    }
    void mult_prog(Program& P, RF& r, const T* X, int N, T* W) {
        T* Xp = wsT((size_t)r.c * N);
        if (r.s == 0) prog_offdiag(P, r.j, X, N, W, Xp);
        else prog_diag_mult(P, r.j, r.s, X, N, W, Xp);
    }

    // state of every block of the batch after the launched passes (one host round trip)
    void rf_readback(std::vector<RF>& R, const RfDev<T>* d_rfd) {
        CK(cudaMemcpyAsync(rf_host, d_rfd, sizeof(RfDev<T>) * R.size(), cudaMemcpyDeviceToHost, stream));
        CK(cudaMemcpyAsync(st_host, d_status + 1, sizeof(int) * 2, cudaMemcpyDeviceToHost, stream));
        sync_stream();
        if (st_host[0]) throw Error(RSC_ERR_TIMEOUT, "a grid barrier wait of the range finder expired");
        if (st_host[1]) throw Error(RSC_ERR_NOT_SPD, "non-finite sample");
        for (size_t i = 0; i < R.size(); ++i) {
            R[i].rank = rf_host[i].rank;
            R[i].active = rf_host[i].active != 0;
        }
    }

    // Alg. 3 for a batch of blocks: samples of up to PREFETCH passes are formed by one
    // implicit product; each pass is one cooperative launch of k_rf_pass, which keeps the
    // stopping decision and the rank on the device, so the host reads the state back
    // only when some block runs out of samples.
    // Blocks small enough for one CTA (m, c <= rfd_max, no power iterations) go through the
    // dense mode; the rest through the batched cooperative passes.
    bool dense_ok(const RF& r) const {
        const int mr = std::min(std::min(r.m, r.c), r.cap);
        return o.power_iters == 0 && mr > 0 && r.m <= rfd_max<T>() && r.c <= rfd_max<T>() &&
               rfd_smem<T>(r.m, r.c, mr) <= RFD_SMEM_CAP;
    }
    void range_finder_batch(std::vector<RF>& R) {
        if (R.empty()) return;
        std::vector<RF> D, B;
        std::vector<int> wd, wb;
        for (size_t i = 0; i < R.size(); ++i) {
            if (dense_ok(R[i])) { D.push_back(R[i]); wd.push_back((int)i); }
            else { B.push_back(R[i]); wb.push_back((int)i); }
        }
        if (!D.empty()) range_finder_dense(D);
        if (!B.empty()) range_finder_batch_coop(B);
        for (size_t i = 0; i < D.size(); ++i) R[wd[i]] = D[i];
        for (size_t i = 0; i < B.size(); ++i) R[wb[i]] = B[i];
    }
    static constexpr size_t RFD_SMEM_CAP = 200 * 1024;
    int* rank_host = nullptr;            // pinned: ranks found by the dense mode
    size_t rank_host_cap = 0;
    std::map<int, T*> ident;             // c x c identities of the current dense batch
    void range_finder_dense(std::vector<RF>& R) {
        ws_reset();
        ident.clear();
        if (R.size() > rank_host_cap) {
            if (rank_host) CK(cudaFreeHost(rank_host));
            rank_host_cap = std::max<size_t>(R.size(), 64);
            CK(cudaMallocHost(&rank_host, sizeof(int) * (rank_host_cap + 2)));
        }
        const double u = sizeof(T) == 8 ? 1.1102230246251565e-16 : 5.9604644775390625e-08;
        int* d_rank = (int*)ws.getb(sizeof(int) * R.size());
        std::vector<Program> progs;
        std::vector<RfDenseTask<T>> tasks;
        size_t smem = 0;
        for (size_t i = 0; i < R.size(); ++i) {
            RF& r = R[i];
            r.maxr = std::min(std::min(r.m, r.c), r.cap);
            T*& X = ident[r.c];
            if (!X) {
                X = wsT((size_t)r.c * r.c);
                k_set_identity<T><<<std::min(cdiv(r.c * r.c, 256), 1024), 256, 0, stream>>>(X, r.c);
                launches++;
            }
            T* Bm = wsT((size_t)r.m * r.c);     // the block, row-major (ld c): B = L X with X = I
            progs.emplace_back();
            mult_prog(progs.back(), r, X, r.c, Bm);
            r.U = lr_alloc((long long)r.c * r.maxr);
            r.V = lr_alloc((long long)r.m * r.maxr);
            tasks.push_back(RfDenseTask<T>{Bm, r.U, r.V, r.m, r.c, r.maxr, 0, r.tol, u, r.block_id,
                                           (uint32_t)restarts << 16, d_rank + i});
            smem = std::max(smem, rfd_smem<T>(r.m, r.c, r.maxr));
            flops += 2.0 * r.m * r.c * r.c;
        }
        run(progs);
        RfDenseTask<T>* dt = (RfDenseTask<T>*)upload_tmp(sTask, tasks);
        PROF(prof, "rf_dense", stream, 0, 0,
             k_rf_dense<T><<<(int)tasks.size(), 512, smem, stream>>>(dt, o.seed, d_status + 2));
        launches++;
        LAUNCH_CHECK();
        CK(cudaMemcpyAsync(rank_host, d_rank, sizeof(int) * R.size(), cudaMemcpyDeviceToHost, stream));
        CK(cudaMemcpyAsync(rank_host + rank_host_cap, d_status + 2, sizeof(int), cudaMemcpyDeviceToHost, stream));
        sync_stream();
        if (rank_host[rank_host_cap]) throw Error(RSC_ERR_NOT_SPD, "non-finite sample");
        // algorithmic work: the range finder on the dense block (three projections and Gram
        // matrices per pass) and V = B U; bytes: the block read once, U and V written once
        double pf = 0, pb = 0;
        for (size_t i = 0; i < R.size(); ++i) {
            RF& r = R[i];
            r.rank = rank_host[i];
            const double f = (double)r.rank * 3.0 * 4.0 * r.c * r.rank + 2.0 * r.m * r.c * r.rank;
            flops += f;
            pf += f;
            pb += sizeof(T) * ((double)r.m * r.c + (double)(r.m + r.c) * r.rank);
        }
        if (prof.enabled("rf_dense")) {
            auto& a = prof.acc["rf_dense" + prof.tag];
            a.flops += pf;
            a.bytes += pb;
        }
    }

    void range_finder_batch_coop(std::vector<RF>& R) {
        if (R.empty()) return;
        ws_reset();
        if (!coop_max) {
            int dev = 0, nsm = 0, per_sm = 0;
            CK(cudaGetDevice(&dev));
            CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
            CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_rf_pass<T>, RFP_THREADS, 0));
            coop_max = std::max(1, std::min(per_sm, 2) * nsm);
            CK(cudaMallocHost(&st_host, sizeof(int) * 2));
        }
        if (R.size() > rf_host_cap) {
            if (rf_host) CK(cudaFreeHost(rf_host));
            rf_host_cap = std::max<size_t>(R.size(), 64);
            CK(cudaMallocHost(&rf_host, sizeof(RfDev<T>) * rf_host_cap));
        }
        const double u = sizeof(T) == 8 ? 1.1102230246251565e-16 : 5.9604644775390625e-08;
        std::vector<int2> chunks;
        bool small = true;   // every block in at most RFP_SMALL chunks: the pass kernel's small-block mode
        for (RF& r : R)
            if (std::min(r.m, r.c) > 0 && cdiv(r.c, RFP_ROWS) > RFP_SMALL) small = false;
        const int halves = small ? 2 : 1;
        for (size_t i = 0; i < R.size(); ++i) {
            RF& r = R[i];
            r.maxr = std::min(std::min(r.m, r.c), r.cap);
            r.rank = 0;
            r.active = r.maxr > 0;
            r.passes = 0;
            r.U = r.maxr ? lr_alloc((long long)r.c * r.maxr) : nullptr;
            r.Y = wsT((size_t)r.c * 16);
            r.Gp = wsT((size_t)std::max(r.m, r.c) * 16 * PREFETCH);
            r.Gb = wsT((size_t)r.m * 16 * PREFETCH);
            r.Yb = wsT((size_t)r.c * 16 * PREFETCH);
            r.pref_base = 0;
            r.pref_n = 0;
            RfDev<T>& d = rf_host[i];
            std::memset(&d, 0, sizeof(d));
            const int nchunk = r.active ? cdiv(r.c, RFP_ROWS) : 0;
            d.U = r.U; d.Y = r.Y;
            d.Z = wsT((size_t)std::max(r.maxr, 1) * 16);
            d.zpart = wsT((size_t)std::max(halves * nchunk * r.maxr, 1) * 16);
            d.gpart = wsT((size_t)std::max(halves * nchunk, 1) * 256);
            d.rinv = wsT(272);
            d.c = r.c; d.maxr = r.maxr; d.nchunk = nchunk;
            d.tol = r.tol; d.u = u;
            d.active = r.active ? 1 : 0;
            for (int q = 0; q < nchunk; ++q) chunks.push_back(make_int2((int)i, q));
        }
        RfDev<T>* d_rfd = (RfDev<T>*)ws.getb(sizeof(RfDev<T>) * R.size());
        CK(cudaMemcpyAsync(d_rfd, rf_host, sizeof(RfDev<T>) * R.size(), cudaMemcpyHostToDevice, stream));
        int2* d_chunks = (int2*)ws.getb(sizeof(int2) * std::max<size_t>(chunks.size(), 1));
        {
            int2* staged = (int2*)upload_tmp(sTask, chunks);
            CK(cudaMemcpyAsync(d_chunks, staged, sizeof(int2) * chunks.size(), cudaMemcpyDeviceToDevice, stream));
        }
        CK(cudaMemsetAsync(d_rfbar, 0, sizeof(unsigned), stream));   // arrival count
        const int nrf = (int)R.size(), nch = (int)chunks.size();
        const int grid = std::max(1, std::min(nch, coop_max));
        for (int t = 0;; ++t) {
            bool any = false, refill = false;
            for (RF& r : R)
                if (r.active) { any = true; refill |= t >= r.pref_base + r.pref_n; }
            if (!any) break;
            if (refill) {
                // samples of passes t .. t + np - 1 are formed together: pass p's block of
                // Y = (L^T L)^q L^T G_p depends only on its own G_p (Philox counter word3 = p).
                // The programs are planned while the passes already launched run; blocks the
                // read-back then shows finished are dropped from the batch.
                std::vector<Program> progs;
                std::vector<RF*> owner;
                for (RF& r : R) {
                    if (!r.active || t < r.pref_base + r.pref_n) continue;
                    // one pass beyond the rank cap holds the adaptive stopping test; the
                    // fixed-rank form (tol = 0) has none
                    const int extra = r.tol > 0 ? 1 : 0;
                    const int np_ = std::min(PREFETCH, std::max(1, cdiv(r.maxr - r.rank, 16) + extra));
                    const int N = 16 * np_;
                    progs.emplace_back();
                    owner.push_back(&r);
                    Program& P = progs.back();
                    Stage& g = next(P);
                    for (int b = 0; b < np_; ++b) {
                        const uint32_t word3 = (uint32_t)(t + b) | ((uint32_t)restarts << 16);
                        for (int r0 = 0; r0 < r.m; r0 += 32)
                            g.gauss.push_back(GaussTask{r.Gb, r.m, r0, r.block_id, word3, N, 16 * b});
                    }
                    mult_T_prog(P, r, r.Gb, N, r.Yb);
                    for (int q = 0; q < o.power_iters; ++q) {
                        mult_prog(P, r, r.Yb, N, r.Gp);
                        mult_T_prog(P, r, r.Gp, N, r.Yb);
                    }
                    r.pref_n = -np_;   // pending: set once the read-back confirms the block
                }
                if (t > 0) {
                    rf_readback(R, d_rfd);
                    bool still = false;
                    for (RF& r : R) still |= r.active;
                    if (!still) break;
                }
                std::vector<Program> keep;
                for (size_t i = 0; i < progs.size(); ++i) {
                    RF& r = *owner[i];
                    const int np_ = -r.pref_n;
                    r.pref_base = t;
                    r.pref_n = np_;
                    if (r.active) keep.push_back(std::move(progs[i]));
                }
                run(keep);
            }
            std::vector<RfPass<T>> pp(R.size(), RfPass<T>{nullptr, 0, 0});
            for (size_t i = 0; i < R.size(); ++i) {
                RF& r = R[i];
                if (!r.active || t >= r.pref_base + r.pref_n) continue;
                pp[i] = RfPass<T>{r.Yb + 16 * (t - r.pref_base), 16 * r.pref_n, t == 0 ? 1 : 0};
                ++r.passes;
            }
            RfPass<T>* d_pp = (RfPass<T>*)upload_tmp(sTask, pp);
            RfBarrier* bar = d_rfbar;
            int* err = d_status + 1;
            int nrf_ = nrf, nch_ = nch;
            unsigned long long* ptime = prof.on ? d_rfp_time : nullptr;
            int small_ = small ? 1 : 0;
            unsigned long long lim = rf_spin_limit;
            void* args[] = {&d_rfd, &d_pp, &nrf_, &d_chunks, &nch_, &bar, &err, &ptime, &small_, &lim};
            PROF(prof, "rf_pass", stream, 0, 0,
                 CK(cudaLaunchCooperativeKernel((const void*)k_rf_pass<T>, dim3(grid), dim3(RFP_THREADS), args, 0,
                                                stream)));
            launches++;
        }
        // algorithmic work of the passes that ran (rank of pass p taken as min(16 p, final rank)):
        // three projections (U^T Y and U Z: U read twice each), three Gram matrices and
        // triangular solves; bytes: the sample block read, U read six times, Q written
        double pf = 0, pb = 0;
        for (RF& r : R) {
            const double c = r.c;
            for (int p = 0; p < r.passes; ++p) {
                const double rk = std::min(16.0 * p, (double)r.rank);
                pf += 3.0 * 4.0 * c * rk * 16 + 3.0 * 2.0 * c * 256 + 3.0 * c * 256;
                pb += sizeof(T) * (c * 16 + 6.0 * c * rk + 2.0 * c * 16);
            }
        }
        flops += pf;
        if (prof.enabled("rf_pass")) {
            auto& a = prof.acc["rf_pass" + prof.tag];
            a.flops += pf;
            a.bytes += pb;
        }
        // V = mult(U): U to row-major, product, back to column-major
        std::vector<Program> progs;
        std::vector<T*> vr(R.size(), nullptr);
        for (size_t i = 0; i < R.size(); ++i) {
            RF& r = R[i];
            if (r.rank == 0) continue;
            progs.emplace_back();
            Program& P = progs.back();
            T* Ur = wsT((size_t)r.c * r.rank);
            vr[i] = wsT((size_t)r.m * r.rank);
            add_copy(next(P), r.U, 1, r.c, Ur, r.rank, 1, r.c, r.rank);
            mult_prog(P, r, Ur, r.rank, vr[i]);
            r.V = lr_alloc((long long)r.m * r.rank);
            add_copy(next(P), vr[i], r.rank, 1, r.V, 1, r.m, r.m, r.rank);
        }
        run(progs);
        sync_stream();   // the workspace is recycled by the next batch
    }

    // ---------------------------------------------------------------- factors of the inverse's off-diagonal blocks
    // For every internal block s of the hierarchical diagonal blocks of one level (Section 4's
    // L^D_j with L21 = V_s U_s^T): tU_s = L_left(s)^{-T} U_s and tV_s = L_right(s)^{-1} V_s by the
    // subtree solves of Alg. 4, all blocks in one staged batch.  Then
    //   (L^D_j)^{-1} x = D^{-1} x - sum_s tV_s (tU_s^T x[cols(s)])  (placed in rows(s)),
    // with D the block diagonal of the leaves: every term reads x, so the preconditioner
    // applies the diagonal solve as three parallel launches instead of the in-order chain.
    void inverse_factors(const std::vector<int>& hier) {
        ws_reset();
        std::vector<Program> progs;
        for (int j : hier) {
            NodeRT& n = nd[j];
            const BlockTree& t = S.tree[j];
            for (int b = 1; b <= t.nblocks; ++b) {
                const int q = n.brank[b];
                if (t.leaf[b] || q == 0) continue;
                const int n1 = t.mid[b] - t.lo[b], n2 = t.hi[b] - t.mid[b];
                {   // tU_b = L_left(b)^{-T} U_b
                    progs.emplace_back();
                    Program& P = progs.back();
                    T* X = wsT((size_t)n1 * q);
                    add_copy(next(P), n.bU[b], 1, n1, X, q, 1, n1, q);
                    prog_diag_solve(P, j, t.left[b], X, q, q, true);
                    n.tU[b] = lr_alloc((long long)n1 * q);
                    add_copy(next(P), X, q, 1, n.tU[b], 1, n1, n1, q);
                }
                {   // tV_b = L_right(b)^{-1} V_b
                    progs.emplace_back();
                    Program& P = progs.back();
                    T* X = wsT((size_t)n2 * q);
                    add_copy(next(P), n.bV[b], 1, n2, X, q, 1, n2, q);
                    prog_diag_solve(P, j, t.right[b], X, q, q, false);
                    n.tV[b] = lr_alloc((long long)n2 * q);
                    add_copy(next(P), X, q, 1, n.tV[b], 1, n2, n2, q);
                }
            }
        }
        run(progs);
        sync_stream();   // the workspace is recycled by the next batch
    }

    // ---------------------------------------------------------------- compressed supernodes of one level
    void compressed_level(const std::vector<int>& comp) {
        std::vector<int> hier;
        int maxnb = 0;
        for (int j : comp)
            if (nd[j].hier) { hier.push_back(j); maxnb = std::max(maxnb, S.tree[j].nblocks); }
        const double t_h0 = now_ms();
        for (int s = 1; s <= maxnb; ++s) {
            std::vector<int> leaves, internals;
            for (int j : hier)
                if (S.tree[j].nblocks >= s) (S.tree[j].leaf[s] ? leaves : internals).push_back(j);
            if (!leaves.empty()) {
                HostTimer ht_(this, "h_leaves");
                // Alg. 6: subtract earlier low-rank blocks p < s (one launch per ancestor depth,
                // since the tiles of one leaf receive several ancestors), then Cholesky
                for (int depth = 0;; ++depth) {
                    std::vector<GemmTask> gt;
                    bool any = false;
                    double gfl = 0, gby = 0;
                    for (int j : leaves) {
                        NodeRT& n = nd[j];
                        const BlockTree& t = S.tree[j];
                        int p = t.parent[s], d = 0;
                        for (; p; p = t.parent[p])
                            if (p < s && n.brank[p] > 0) { if (d == depth) break; ++d; }
                        if (!p) continue;
                        any = true;
                        const int sz = t.hi[s] - t.lo[s], mp = t.hi[p] - t.mid[p];
                        const T* Vp = n.bV[p] + (t.lo[s] - t.mid[p]);
                        T* Ls = arena + n.leaf_off[s];
                        for (int c0 = 0; c0 < sz; c0 += TILE)
                            for (int r0 = c0; r0 < sz; r0 += TILE) {
                                GemmTask g{};
                                g.A = Vp + r0; g.B = Vp + c0; g.C = Ls + r0 + (size_t)c0 * sz;
                                g.lda = mp; g.ldb = mp; g.ldc = sz;
                                g.m = std::min(TILE, sz - r0); g.n = std::min(TILE, sz - c0);
                                g.K = n.brank[p]; g.moff = r0 - c0; g.lower = r0 == c0;
                                gt.push_back(g);
                            }
                        flops += (double)sz * (sz + 1) * n.brank[p];
                        gfl += (double)sz * (sz + 1) * n.brank[p];
                        gby += sizeof(T) * ((double)sz * n.brank[p] + (double)sz * (sz + 1));
                    }
                    if (!any) break;
                    GemmTask* dg = (GemmTask*)upload_tmp(sT2, gt);
                    PROF(prof, "leaf_gemm", stream, gfl, gby, k_gemm_tile<T><<<(int)gt.size(), 256, 0, stream>>>(dg));
                    launches++;
                    LAUNCH_CHECK();
                }
                std::vector<DensePanel> dp;
                std::vector<PotrfTask> lt;
                size_t lsm = 0;
                bool fused = true;   // every leaf fits one CTA's shared memory: one launch for all
                for (int j : leaves) {
                    const BlockTree& t = S.tree[j];
                    const int sz = t.hi[s] - t.lo[s];
                    dp.push_back(DensePanel{arena + nd[j].leaf_off[s], sz, sz, sz, j});
                    lt.push_back(PotrfTask{arena + nd[j].leaf_off[s], sz, sz, j});
                    const size_t need = leaf_smem(sz);
                    if (sz > LEAF_FUSED_MAX || need > LEAF_SMEM_CAP) fused = false;
                    lsm = std::max(lsm, need);
                }
                if (fused) {
                    double fl = 0, by = 0;
                    for (auto& x : lt) {
                        fl += (double)x.nb * x.nb * x.nb / 3.0;
                        by += sizeof(T) * (double)x.nb * (x.nb + 1);   // lower triangle read and written
                    }
                    flops += fl;
                    PotrfTask* dl = (PotrfTask*)upload_tmp(sTask, lt);
                    PROF(prof, "leaf_factor", stream, fl, by,
                         k_leaf_factor<T><<<(int)lt.size(), 256, lsm, stream>>>(dl, d_status));
                    launches++;
                    LAUNCH_CHECK();
                } else {
                    factor_dense_batch(dp);
                }
                std::vector<TrsvTask> tv;
                for (int j : leaves) {
                    const BlockTree& t = S.tree[j];
                    const int sz = t.hi[s] - t.lo[s];
                    tv.push_back(TrsvTask{arena + nd[j].leaf_off[s], sz, sz, sz, invs + nd[j].leaf_inv[s], sz, 2});
                }
                launch_inverses(tv);
            }
            if (!internals.empty()) {
                HostTimer ht_(this, "h_internal_rf");
                std::vector<RF> R;
                for (int j : internals) {
                    const BlockTree& t = S.tree[j];
                    RF r;
                    r.j = j; r.s = s;
                    r.m = t.hi[s] - t.mid[s];
                    r.c = t.mid[s] - t.lo[s];
                    r.tol = fixed ? 0.0 : tol_D;
                    if (fixed) r.cap = rank_heuristic(r.m, r.c, fr_cur.alpha_D, fr_cur.p);
                    r.block_id = ((uint32_t)j << 12) | (uint32_t)s;
                    R.push_back(r);
                }
                range_finder_batch(R);
                for (RF& r : R) {
                    NodeRT& n = nd[r.j];
                    n.bV[s] = r.V; n.bU[s] = r.U; n.brank[s] = r.rank;
                }
            }
        }
        if (!hier.empty()) inverse_factors(hier);
        if (prof.on && maxnb) { sync_stream(); prof.wall("wall_hier_diag", now_ms() - t_h0); }
        const double t_o0 = now_ms();
        std::vector<RF> R;
        for (int j : comp)
            if (nd[j].r > 0) {
                RF r;
                r.j = j; r.s = 0;
                r.m = nd[j].r; r.c = nd[j].c;
                r.tol = fixed ? 0.0 : tol;
                if (fixed) r.cap = rank_heuristic(r.m, r.c, fr_cur.alpha_O, fr_cur.p);
                r.block_id = (uint32_t)j << 12;
                R.push_back(r);
            }
        range_finder_batch(R);
        for (RF& r : R) {
            NodeRT& n = nd[r.j];
            n.V = r.V; n.U = r.U; n.rank = r.rank;
        }
        for (int j : comp) h_lo[j] = LoOp{nd[j].V, std::max(nd[j].r, 1), nd[j].rank};
        if (prof.on) prof.wall("wall_offdiag_rf", now_ms() - t_o0);
    }

    void check_status() {
        int st[3] = {0, 0, 0};
        CK(cudaMemcpyAsync(st, d_status, sizeof(int) * 3, cudaMemcpyDeviceToHost, stream));
        sync_stream();
        if (st[1]) throw Error(RSC_ERR_TIMEOUT, "a bounded device wait expired");
        if (st[2]) throw Error(RSC_ERR_NOT_SPD, "non-finite sample");
        if (st[0]) throw Error(RSC_ERR_NOT_SPD, "indefinite diagonal block in supernode " + std::to_string(st[0] - 1));
    }

    // ---------------------------------------------------------------- factor
    // ---------------------------------------------------------------- per-level launches
    // dense panel factorization steps of the level and the inverses of its dense diagonal blocks
    void issue_panels_and_inverses(int l) {
        run_panel_steps(panel_steps[l]);
        if (inv_count[l]) {
            double fl = 0;
            for (int j : S.level_nodes[l])
                if (!nd[j].hier) fl += (double)nd[j].c * std::min(nd[j].c, SOLVE_MAX) * std::min(nd[j].c, SOLVE_MAX) / 3.0;
            const dim3 grid((unsigned)inv_count[l], (unsigned)cdiv(inv_maxc[l], TRSV_CW));
            PROF(prof, "trinv", stream, fl, 0, k_trsv_subst<T, TRSV_CW><<<grid, 256, 0, stream>>>(inv_tasks[l]));
            launches++;
            LAUNCH_CHECK();
        }
    }
    // algorithmic flops of the level's dense work (counted whether launched or replayed)
    void count_level_flops(int l) {
        for (int j : S.level_nodes[l]) {
            const NodeRT& n = nd[j];
            if (!n.hier) flops += (double)n.c * std::min(n.c, SOLVE_MAX) * std::min(n.c, SOLVE_MAX) / 3.0;
            if (!n.compressed) {
                const double c = n.c, r = n.r;
                flops += c * c * c / 3.0 + r * c * c;
            }
        }
    }
    // the level's extend-add into its ancestors (d_lo holds the sources' L^O_k or V_k)
    void issue_push(int l) {
        if (!push_count[l]) return;
        double pf = 0, pb = 0;
        if (prof.on)
            for (auto& e : push_elems[l]) {
                pf += 2.0 * e.elems * h_lo[e.k].K;
                pb += sizeof(T) * ((double)e.rows * h_lo[e.k].K + 2.0 * e.elems);
            }
        if (tc && push_count_tc[l]) {
            auto kern = tc_tf32 ? k_push_tc<true> : k_push_tc<false>;
            const int pad = tc_tf32 ? TC_PAD_SMEM_TF32 : TC_PAD_SMEM;
            PROF(prof, "push_tc", stream, pf, pb,
                 kern<<<push_count_tc[l], 128, pad, stream>>>(
                     push_tasks_tc[l], d_lo, d_tgt, d_rows, d_rows_ptr, d_leaf, (float*)arena, d_status + 1));
        } else {
            PROF(prof, "push", stream, pf, pb,
                 k_push<T><<<push_count[l], 256, 0, stream>>>(push_tasks[l], d_lo, d_tgt, d_rows, d_rows_ptr, d_leaf,
                                                             arena));
        }
        launches++;
        LAUNCH_CHECK();
    }
    int dense_prefix = 0;                       // levels before the first compressed supernode
    cudaGraphExec_t dense_graph = nullptr;      // their launches, captured once per plan
    long long dense_graph_launches = 0;

    void run_once(const double* val) {
        lr_used = 0;
        flops = 0.0;
        CK(cudaMemsetAsync(d_status, 0, sizeof(int) * 3, stream));
        CK(cudaMemsetAsync(arena, 0, sizeof(T) * std::max<long long>(arena_elems, 1), stream));
        const size_t nval = (size_t)(S.lsrc.empty() ? 0 : *std::max_element(S.lsrc.begin(), S.lsrc.end()) + 1);
        if (vals_dev) CK(cudaMemcpyAsync(d_valbuf, d_uval, sizeof(double) * nval, cudaMemcpyDeviceToDevice, stream));
        else CK(cudaMemcpyAsync(d_valbuf, val, sizeof(double) * nval, cudaMemcpyHostToDevice, stream));
        if (asm_cnt) {
            k_assemble<T><<<std::min(cdiv(asm_cnt, 256), 8192), 256, 0, stream>>>(d_valbuf, d_asm_src, d_asm_dst, asm_cnt,
                                                                                   arena);
            launches++;
        }
        if (vals_dev) {   // sparse-block values gathered on the device
            if (!sp_src.empty()) {
                k_gather_vals<<<std::min(cdiv((long long)sp_src.size(), 256), 4096), 256, 0, stream>>>(
                    d_uval, d_spsrc, (long long)sp_src.size(), d_spval);
                launches++;
            }
        } else {
            std::vector<double> spv(sp_src.size());
            for (size_t e = 0; e < sp_src.size(); ++e) spv[e] = val[sp_src[e]];
            if (!spv.empty())
                CK(cudaMemcpyAsync(d_spval, spv.data(), sizeof(double) * spv.size(), cudaMemcpyHostToDevice, stream));
            CK(cudaStreamSynchronize(stream));
        }
        for (int j = 0; j < S.M; ++j) {
            NodeRT& n = nd[j];
            n.rank = 0; n.V = n.U = nullptr;
            if (n.hier) {
                std::fill(n.brank.begin(), n.brank.end(), 0);
                std::fill(n.bV.begin(), n.bV.end(), nullptr);
                std::fill(n.bU.begin(), n.bU.end(), nullptr);
                std::fill(n.tV.begin(), n.tV.end(), nullptr);
                std::fill(n.tU.begin(), n.tU.end(), nullptr);
            }
            if (n.compressed) h_lo[j] = LoOp{nullptr, 1, 0};
        }
        // levels before the first compressed supernode have a launch list fixed by the plan: one
        // CUDA graph (captured at the first factorization with this plan) replays them
        int l_start = 0;
        if (dense_prefix > 0 && !prof.on && !no_graph) {
            CK(cudaMemcpyAsync(d_lo, h_lo.data(), sizeof(LoOp) * S.M, cudaMemcpyHostToDevice, stream));
            if (!dense_graph) {
                const long long before = launches;
                CK(cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal));
                for (int l = 0; l < dense_prefix; ++l) {
                    issue_panels_and_inverses(l);
                    issue_push(l);
                }
                cudaGraph_t g = nullptr;
                CK(cudaStreamEndCapture(stream, &g));
                CK(cudaGraphInstantiate(&dense_graph, g, 0));
                CK(cudaGraphDestroy(g));
                dense_graph_launches = launches - before;
                launches = before;
            }
            CK(cudaGraphLaunch(dense_graph, stream));
            launches += dense_graph_launches;
            for (int l = 0; l < dense_prefix; ++l) count_level_flops(l);
            l_start = dense_prefix;
        }
        for (int l = l_start; l < S.nlevels; ++l) {
            const double t_l0 = now_ms();
            if (std::getenv("RSC_PROFILE_BY_LEVEL")) {
                char tg[16];
                std::snprintf(tg, sizeof(tg), "@%02d", l);
                prof.tag = tg;
            }
            issue_panels_and_inverses(l);
            count_level_flops(l);
            std::vector<int> comp;
            for (int j : S.level_nodes[l])
                if (nd[j].compressed) comp.push_back(j);
            if (!comp.empty()) {
                check_status();
                compressed_level(comp);
            }
            // extend-add of the level into its ancestors
            CK(cudaMemcpyAsync(d_lo, h_lo.data(), sizeof(LoOp) * S.M, cudaMemcpyHostToDevice, stream));
            issue_push(l);
            ib_dense_level(l);
            sync_stream();   // h_lo is rewritten by the next level
            if (prof.on) {
                char nm[32];
                std::snprintf(nm, sizeof(nm), "wall_level%02d", l);
                prof.wall(nm, now_ms() - t_l0);
            }
        }
        // push flops: lower half of L^O_k L^O_k^T per source
        for (int k = 0; k < S.M; ++k) {
            const double rk = nd[k].r, K = h_lo[k].K;
            flops += rk * (rk + 1) * K;
        }
        prof.tag.clear();
        check_status();
    }

    rsc_status factor(const double* val, double tol_in, const FixedRank* fr) override {
        is_factored = false;
        // the records of the allocation-free apply point into the factor being replaced
        na_y = nullptr;
        na_loaded_gen = -1;
        plan1.clear();   // launch lists of the previous factor: their memory is released now
        planN.clear();
        fixed = fr != nullptr;
        if (fixed) fr_cur = *fr;
        tol = fixed ? 0.0 : (tol_in > 0 ? tol_in : 0.0);
        tol_D = tol;
        const bool compress = fixed || tol > 0;
        diag_on = compress && o.diag_compress;
        restarts = 0;
        cudaEvent_t e0, e1;
        CK(cudaEventCreate(&e0));
        CK(cudaEventCreate(&e1));
        launches = 0;
        prof.flush();
        prof.mark();
        if (prof.on) {
            if (!d_rfp_time) CK(cudaMalloc(&d_rfp_time, sizeof(unsigned long long) * 16));
            CK(cudaMemsetAsync(d_rfp_time, 0, sizeof(unsigned long long) * 16, stream));
        }
        // the first factorization of a BF16 / TF32 handle tunes the thin products' kernel variants
        tuner.tuning = tc && !tuned_once;
        // the timed region covers every attempt: a restart (Section 5.3) repeats the factorization
        CK(cudaEventRecord(e0, stream));
        for (;;) {
            if (!have_plan || plan_compress != compress || plan_diag != diag_on) build_plan(compress, diag_on);
            try {
                run_once(val);
            } catch (const Error& e) {
                if (e.status != RSC_ERR_NOT_SPD || !diag_on) {
                    cudaEventDestroy(e0);
                    cudaEventDestroy(e1);
                    tuner.abandon();
                    throw;
                }
                sync_stream();
                prof.flush();
                ++restarts;
                if (restarts > o.max_restarts) diag_on = false;
                else if (fixed) fr_cur.alpha_D *= 1.25;   // Section 5.3
                else tol_D /= 1.25;
                continue;
            }
            break;
        }
        // the launch lists of the preconditioner apply are built at their first use (inside the
        // solve's timed region): one column for rsc_solve, N columns for the batched solve
        ++factor_gen;
        CK(cudaEventRecord(e1, stream));
        CK(cudaEventSynchronize(e1));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        factor_seconds = ms * 1e-3;
        if (tuner.tuning) { tuner.finish(); tuned_once = true; }
        prof.flush();
        if (prof.on && d_rfp_time) {
            unsigned long long tp[16];
            CK(cudaMemcpy(tp, d_rfp_time, sizeof(tp), cudaMemcpyDeviceToHost));
            static const char* names[13] = {"rfp_A_copy_tn", "rfp_B_red", "rfp_C_nn_tn", "rfp_D_red", "rfp_E_nn_gram",
                                            "rfp_F_test_chol", "rfp_G_rinv_tn", "rfp_H_red", "rfp_I_nn_gram",
                                            "rfp_J_chol", "rfp_K_rinv_gram", "rfp_L_chol", "rfp_M_rinv_store"};
            for (int i = 0; i < 13; ++i) prof.wall(names[i], tp[i] * 1e-6);
        }
        is_factored = true;
        return RSC_OK;
    }

    // ---------------------------------------------------------------- preconditioner apply
    // The apply is a fixed list of batched launches built once per factor:
    //   forward, level by level: dense diagonal solves (TRSV, all small nodes of the
    //   level in one launch), the in-order actions of hierarchical / large dense
    //   diagonal blocks batched across the level's nodes by action index, then the
    //   off-diagonal updates y_R -= L^O y_C (or V (U^T y_C));
    //   backward, levels in reverse: y_C -= L^O^T y_R (or U (V^T y_R)), the actions
    //   in reverse order, the transposed small dense solves.
    // It is captured once into a CUDA graph reading g_in and writing g_out.
    enum LKind { L_PERM_IN, L_PERM_OUT, L_TRSV, L_TN, L_NN, L_HSOLVE, L_COPY, L_CSR };
    struct Launch { int kind; int count; size_t off; int flag; };
    // one launch list (and its CUDA graph) per number of right-hand sides: plan1 for the PCG of
    // one system, planN for the batched PCG (N columns of y, row-major)
    struct ApplyPlan {
        int N = 1;
        std::vector<Launch> seq;
        DeviceMem mem;
        T* y = nullptr;
        T* tmp = nullptr;
        double* gin = nullptr;
        double* gout = nullptr;
        HTask* hs = nullptr;
        HAct* hacts = nullptr;
        TrsvTask* trsv = nullptr;
        TnTask* tn = nullptr;
        NnTask* nn = nullptr;
        CopyTask* copy = nullptr;        // interior blocks (Section 5.1)
        CsrTask* csr = nullptr;
        T* y2 = nullptr;                 // second work vector: the interior blocks' solves
        cudaGraphExec_t graph = nullptr;
        long long gen = -1;              // factorization the plan was built for
        double flops = 0, bytes = 0;
        void clear() {   // the plan's device blocks are kept for its rebuild (DeviceMem::recycle)
            if (graph) cudaGraphExecDestroy(graph);
            graph = nullptr;
            mem.recycle();
            seq.clear();
            flops = bytes = 0;
            gen = -1;
        }
    };
    ApplyPlan plan1, planN;
    ApplyPlan* pl = &plan1;              // the plan being built

    struct SolveBuild {
        std::vector<TrsvTask> trsv;
        std::vector<TnTask> tn;
        std::vector<NnTask> nn;
        std::vector<CopyTask> copy;
        std::vector<CsrTask> csr;
    };
    struct Act { std::vector<TrsvTask> trsv; std::vector<TnTask> tn; std::vector<NnTask> nn; };

    static void push_nn_chunks(std::vector<NnTask>& v, NnTask t) {
        for (int r0 = 0; r0 < t.nrow; r0 += NN_ROWS) { NnTask c = t; c.row0 = r0; v.push_back(c); }
    }
    // columns of A per apply TN task: the vector kernel k_tn1 takes 32, the staged k_tn_s (several
    // right-hand sides) 64
    int ap_tn_cols() const { return pl->N == 1 ? TN_COLS : TS_COLS; }
    void push_tn_chunks(std::vector<TnTask>& v, const TnTask& t) const {
        for (int t0 = 0; t0 < t.K; t0 += ap_tn_cols()) { TnTask c = t; c.t0 = t0; v.push_back(c); }
    }
    // vector forms on y (ld 1, one column); yoff / ymap index rows of y
    TnTask vtn(const void* A, int lda, int K, int nrow, const int32_t* ymap, int yoff, T* Z, double alpha = 1.0,
               double beta = 0.0) {
        return tn_task(A, lda, K, nrow, nullptr, 0, ymap, yoff, pl->y, pl->N, Z, pl->N, pl->N, alpha, beta);
    }
    NnTask vnn(const void* A, int lda, int K, int nrow, const int32_t* ymap, int yoff, const T* Z, bool atomic) {
        return nn_task(A, lda, K, nrow, nullptr, 0, ymap, yoff, Z, pl->N, pl->y, pl->N, pl->N, -1.0, atomic);
    }

    // In-order actions of one diagonal block (vector right-hand side, rows c0.. of y).
    void diag_actions(int j, bool transpose, T*& zcur, std::vector<Act>& acts) {
        const NodeRT& n = nd[j];
        const int N = pl->N;
        T* X = pl->y + n.c0 * N;
        if (!n.hier) {
            const T* L = arena + n.off;
            const int ld = n.ld, c = n.c, bs = SOLVE_MAX;
            const int nblk = cdiv(c, bs);
            for (int bi = 0; bi < nblk; ++bi) {
                const int b = transpose ? nblk - 1 - bi : bi;
                const int b0 = b * bs, b1 = std::min(c, b0 + bs);
                Act a;
                a.trsv.push_back(TrsvTask{inv_block(j, b0), b1 - b0, b1 - b0, N, X + (size_t)b0 * N, N, transpose ? 1 : 0});
                if (!transpose && b1 < c)
                    push_nn_chunks(a.nn, vnn(L + b1 + (size_t)b0 * ld, ld, b1 - b0, c - b1, nullptr, (int)(n.c0 + b1),
                                             X + (size_t)b0 * N, false));
                if (transpose && b0 > 0)   // y[c0 : c0+b0] -= L[b0:b1, 0:b0]^T y[c0+b0 : c0+b1]
                    push_tn_chunks(a.tn, vtn(L + b0, ld, b0, b1 - b0, nullptr, (int)(n.c0 + b0), X, -1.0, 1.0));
                acts.push_back(std::move(a));
            }
            return;
        }
        const BlockTree& t = S.tree[j];
        std::function<void(int)> rec = [&](int s) {
            if (t.leaf[s]) {
                Act a;
                const int sz = t.hi[s] - t.lo[s];
                a.trsv.push_back(TrsvTask{invs + n.leaf_inv[s], sz, sz, N, X + (size_t)t.lo[s] * N, N, transpose ? 1 : 0});
                acts.push_back(std::move(a));
                return;
            }
            const int n1 = t.mid[s] - t.lo[s], n2 = t.hi[s] - t.mid[s], q = n.brank[s];
            auto lowrank = [&]() {
                if (!q) return;
                Act a;
                T* Z = zcur;
                zcur += (size_t)q * N;
                if (!transpose) {   // X2 -= V_s (U_s^T X1)
                    push_tn_chunks(a.tn, vtn(n.bU[s], n1, q, n1, nullptr, (int)(n.c0 + t.lo[s]), Z));
                    push_nn_chunks(a.nn, vnn(n.bV[s], n2, q, n2, nullptr, (int)(n.c0 + t.mid[s]), Z, false));
                } else {            // X1 -= U_s (V_s^T X2)
                    push_tn_chunks(a.tn, vtn(n.bV[s], n2, q, n2, nullptr, (int)(n.c0 + t.mid[s]), Z));
                    push_nn_chunks(a.nn, vnn(n.bU[s], n1, q, n1, nullptr, (int)(n.c0 + t.lo[s]), Z, false));
                }
                acts.push_back(std::move(a));
            };
            if (!transpose) { rec(t.left[s]); lowrank(); rec(t.right[s]); }
            else { rec(t.right[s]); lowrank(); rec(t.left[s]); }
        };
        rec(t.root);
    }

    void build_solve_plan(int N = 1) {
        pl = N == 1 ? &plan1 : &planN;
        pl->clear();
        pl->N = N;
        pl->gen = factor_gen;
        const long long n = S.n;
        pl->y = (T*)pl->mem.alloc(sizeof(T) * n * N);
        pl->gin = (double*)pl->mem.alloc(sizeof(double) * n * N);
        pl->gout = (double*)pl->mem.alloc(sizeof(double) * n * N);
        long long tmp_total = 0;
        for (int j = 0; j < S.M; ++j) {
            const NodeRT& nn = nd[j];
            tmp_total += nn.compressed ? nn.rank : 0;
            if (nn.hier)
                for (int b = 1; b <= S.tree[j].nblocks; ++b) tmp_total += 2 * nn.brank[b];
        }
        tmp_total *= N;
        pl->tmp = (T*)pl->mem.alloc(sizeof(T) * std::max<long long>(tmp_total, 1));
        T* zcur = pl->tmp;
        SolveBuild B;
        auto emit = [&](int kind, size_t off, size_t cnt, int flag) {
            if (cnt) pl->seq.push_back(Launch{kind, (int)cnt, off, flag});
        };
        auto emit_acts = [&](std::vector<std::vector<Act>>& per_node) {
            size_t maxa = 0;
            for (auto& v : per_node) maxa = std::max(maxa, v.size());
            for (size_t ai = 0; ai < maxa; ++ai) {
                size_t o1 = B.trsv.size(), o2 = B.tn.size(), o3 = B.nn.size();
                for (auto& v : per_node) {
                    if (ai >= v.size()) continue;
                    Act& a = v[ai];
                    B.trsv.insert(B.trsv.end(), a.trsv.begin(), a.trsv.end());
                    B.tn.insert(B.tn.end(), a.tn.begin(), a.tn.end());
                    B.nn.insert(B.nn.end(), a.nn.begin(), a.nn.end());
                }
                emit(L_TRSV, o1, B.trsv.size() - o1, 0);
                emit(L_TN, o2, B.tn.size() - o2, 0);
                emit(L_NN, o3, B.nn.size() - o3, 0);
            }
        };
        // persistent solves: actions and tasks (acts as offsets until upload)
        std::vector<HAct> HA;
        std::vector<HTask> HT;
        auto emit_hsolve = [&](std::vector<int>& nodes, bool transpose, std::vector<std::vector<Act>>& rest) {
            size_t o = HT.size();
            int maxc = 0;
            for (int j : nodes) {
                const NodeRT& nn = nd[j];
                if (pick_cw(nn.c) == 0) { rest.emplace_back(); T* zc = zcur; diag_actions(j, transpose, zc, rest.back()); zcur = zc; continue; }
                const long long first = (long long)HA.size();
                const double keep = flops;
                hacts(j, 0, transpose, HA);
                flops = keep;
                HT.push_back(HTask{(const HAct*)(intptr_t)first, (long long)HA.size() - first, pl->y + nn.c0 * N, N, N, nn.c,
                                   transpose ? 1 : 0});
                maxc = std::max(maxc, nn.c);
            }
            if (HT.size() > o) pl->seq.push_back(Launch{L_HSOLVE, (int)(HT.size() - o), o, maxc});
        };
        // Section 5.1: an interior block's part of the forward substitution ends with
        // y[R_B] -= A(R_B, C_B) L_B^{-T} y[C_B]; the backward one starts with
        // y[C_B] -= L_B^{-1} A(C_B, R_B) y[R_B]; both solves with L_B run on the second vector y2
        // (rows C_B), the block's supernodes level by level as in the main sweep.
        if (ib_on) pl->y2 = (T*)pl->mem.alloc(sizeof(T) * n * N);
        auto ib_solve = [&](const std::vector<int>& bl, int top, bool transpose) {
            T* keep = pl->y;
            pl->y = pl->y2;
            for (int li = 0; li <= top; ++li) {
                const int lv = transpose ? top - li : li;
                std::vector<int> nodes;
                for (int b : bl)
                    if (lv < (int)iblocks[b].lvl.size())
                        nodes.insert(nodes.end(), iblocks[b].lvl[lv].begin(), iblocks[b].lvl[lv].end());
                if (nodes.empty()) continue;
                if (transpose) {   // y2[C_k] -= L(R_k in C_B, C_k)^T y2[R_k in C_B]
                    const size_t o2 = B.tn.size();
                    for (int j : nodes) {
                        const NodeRT& nn = nd[j];
                        if (nn.r == 0) continue;
                        push_tn_chunks(B.tn, vtn(arena + nn.off + nn.c, nn.ld, nn.c, nn.r, d_rows + S.rows_ptr[j], 0,
                                                 pl->y + nn.c0 * N, -1.0, 1.0));
                        pl->bytes += sizeof(T) * (double)nn.r * nn.c;
                    }
                    emit(L_TN, o2, B.tn.size() - o2, 0);
                }
                std::vector<std::vector<Act>> acts;
                std::vector<int> big;
                const size_t o = B.trsv.size();
                for (int j : nodes) {
                    const NodeRT& nn = nd[j];
                    pl->bytes += sizeof(T) * ((double)nn.c * (nn.c + 1) / 2);
                    if (nn.c <= SOLVE_MAX)
                        B.trsv.push_back(TrsvTask{inv_block(j, 0), nn.c, nn.c, N, pl->y + nn.c0 * N, N, transpose ? 1 : 0});
                    else big.push_back(j);
                }
                emit(L_TRSV, o, B.trsv.size() - o, 0);
                emit_hsolve(big, transpose, acts);
                emit_acts(acts);
                if (!transpose) {   // y2[R_k in C_B] -= L(R_k in C_B, C_k) y2[C_k]
                    const size_t o3 = B.nn.size();
                    for (int j : nodes) {
                        const NodeRT& nn = nd[j];
                        if (nn.r == 0) continue;
                        push_nn_chunks(B.nn, vnn(arena + nn.off + nn.c, nn.ld, nn.c, nn.r, d_rows + S.rows_ptr[j], 0,
                                                 pl->y + nn.c0 * N, true));
                        pl->bytes += sizeof(T) * (double)nn.r * nn.c;
                    }
                    emit(L_NN, o3, B.nn.size() - o3, 0);
                }
            }
            pl->y = keep;
        };
        auto ib_csr = [&](const IbCsr& c, const T* X, T* Y, double alpha, int mode) {
            for (int r0 = 0; r0 < c.blk.nrows; r0 += 16) {
                CsrTask t{c.blk, X, N, Y, N, N, r0, alpha};
                t.rmap = c.rmap;
                t.mode = mode;
                B.csr.push_back(t);
            }
        };
        auto ib_forward = [&](int l) {
            if (!ib_on || ib_root[l].empty()) return;
            const std::vector<int>& bl = ib_root[l];
            size_t oc = B.copy.size();
            for (int b : bl) {   // y2[C_B] = y[C_B]
                const IBlock& Bk = iblocks[b];
                const long long m = (Bk.c1 - Bk.c0) * N;
                B.copy.push_back(CopyTask{pl->y + Bk.c0 * N, 1, 0, pl->y2 + Bk.c0 * N, 1, 0, (int)m, 1, 0});
            }
            emit(L_COPY, oc, B.copy.size() - oc, 0);
            ib_solve(bl, l, true);
            const size_t os = B.csr.size();
            for (int b : bl) ib_csr(iblocks[b].fwd, pl->y2, pl->y, -1.0, 2);   // y[R_B] -= A(R_B, C_B) y2[C_B]
            emit(L_CSR, os, B.csr.size() - os, 0);
        };
        auto ib_backward = [&](int l) {
            if (!ib_on || ib_root[l].empty()) return;
            const std::vector<int>& bl = ib_root[l];
            size_t oc = B.copy.size();
            for (int b : bl) {   // y2[C_B] = 0
                const IBlock& Bk = iblocks[b];
                B.copy.push_back(CopyTask{d_zero, 0, 0, pl->y2 + Bk.c0 * N, 1, 0, (int)((Bk.c1 - Bk.c0) * N), 1, 0});
            }
            emit(L_COPY, oc, B.copy.size() - oc, 0);
            const size_t os = B.csr.size();
            for (int b : bl) ib_csr(iblocks[b].bwd, pl->y, pl->y2, 1.0, 0);   // y2[C_B] = A(C_B, R_B) y[R_B]
            emit(L_CSR, os, B.csr.size() - os, 0);
            ib_solve(bl, l, false);
            oc = B.copy.size();
            for (int b : bl) {   // y[C_B] -= y2[C_B]
                const IBlock& Bk = iblocks[b];
                const long long m = (Bk.c1 - Bk.c0) * N;
                B.copy.push_back(CopyTask{pl->y2 + Bk.c0 * N, 1, 0, pl->y + Bk.c0 * N, 1, 0, (int)m, 1, 1});
            }
            emit(L_COPY, oc, B.copy.size() - oc, 0);
        };
        emit(L_PERM_IN, 0, 1, 0);
        std::vector<std::vector<T*>> ztmp(S.nlevels);
        // hierarchical diagonal blocks through the factors of their inverse: per level, the
        // low-rank products z_s = tU_s^T y[cols(s)] (TN) before the leaf solves (TRSV, in place),
        // then y[rows(s)] -= tV_s z_s (NN, atomic: the row ranges of nested blocks overlap);
        // the transpose exchanges the roles of tU and tV.  z_s is kept per block.
        std::map<std::pair<int, int>, T*> hz;
        auto hier_terms = [&](int j, bool transpose, std::vector<TnTask>& tn, std::vector<NnTask>& nnv) {
            const NodeRT& nn = nd[j];
            const BlockTree& t = S.tree[j];
            for (int b = 1; b <= t.nblocks; ++b) {
                const int q = nn.brank[b];
                if (t.leaf[b] || q == 0) continue;
                const int n1 = t.mid[b] - t.lo[b], n2 = t.hi[b] - t.mid[b];
                T*& z = hz[{j, b}];
                if (!z) { z = zcur; zcur += (size_t)q * N; }
                if (!transpose) {
                    push_tn_chunks(tn, vtn(nn.tU[b], n1, q, n1, nullptr, (int)(nn.c0 + t.lo[b]), z));
                    push_nn_chunks(nnv, vnn(nn.tV[b], n2, q, n2, nullptr, (int)(nn.c0 + t.mid[b]), z, true));
                } else {
                    push_tn_chunks(tn, vtn(nn.tV[b], n2, q, n2, nullptr, (int)(nn.c0 + t.mid[b]), z));
                    push_nn_chunks(nnv, vnn(nn.tU[b], n1, q, n1, nullptr, (int)(nn.c0 + t.lo[b]), z, true));
                }
                pl->bytes += sizeof(T) * (double)q * (n1 + n2);
            }
        };
        auto hier_leaves = [&](int j, bool transpose) {
            const NodeRT& nn = nd[j];
            const BlockTree& t = S.tree[j];
            for (int b = 1; b <= t.nblocks; ++b)
                if (t.leaf[b]) {
                    const int sz = t.hi[b] - t.lo[b];
                    B.trsv.push_back(
                        TrsvTask{invs + nn.leaf_inv[b], sz, sz, N, pl->y + (nn.c0 + t.lo[b]) * N, N, transpose ? 1 : 0});
                    pl->bytes += sizeof(T) * (double)sz * sz;
                }
        };
        for (int l = 0; l < S.nlevels; ++l) {
            std::vector<std::vector<Act>> acts;
            std::vector<int> big;
            std::vector<NnTask> hnn;
            size_t oh = B.tn.size();
            for (int j : S.level_nodes[l])
                if (nd[j].hier) hier_terms(j, false, B.tn, hnn);
            emit(L_TN, oh, B.tn.size() - oh, 0);
            size_t o = B.trsv.size();
            for (int j : S.level_nodes[l]) {
                const NodeRT& nn = nd[j];
                if (nn.hier) { hier_leaves(j, false); continue; }
                pl->bytes += 2.0 * sizeof(T) * ((double)nn.c * (nn.c + 1) / 2);
                if (nn.c <= SOLVE_MAX)
                    B.trsv.push_back(TrsvTask{inv_block(j, 0), nn.c, nn.c, N, pl->y + nn.c0 * N, N, 0});
                else big.push_back(j);
            }
            emit(L_TRSV, o, B.trsv.size() - o, 0);
            size_t ohn = B.nn.size();
            B.nn.insert(B.nn.end(), hnn.begin(), hnn.end());
            emit(L_NN, ohn, hnn.size(), 0);
            emit_hsolve(big, false, acts);
            emit_acts(acts);
            size_t o2 = B.tn.size(), o3 = B.nn.size();
            for (int j : S.level_nodes[l]) {
                const NodeRT& nn = nd[j];
                if (nn.r == 0) continue;
                const int32_t* Rj = d_rows + S.rows_ptr[j];
                if (!nn.compressed) {   // y_R -= L^O_j y_C (atomic: nodes of a level share rows of R)
                    push_nn_chunks(B.nn, vnn(arena + nn.off + nn.c, nn.ld, nn.c, nn.r, Rj, 0, pl->y + nn.c0 * N, true));
                    pl->bytes += 2.0 * sizeof(T) * nn.r * nn.c;
                } else if (nn.rank) {   // y_R -= V_j (U_j^T y_C)
                    T* tmp = zcur; zcur += (size_t)nn.rank * N;
                    ztmp[l].push_back(tmp);
                    push_tn_chunks(B.tn, vtn(nn.U, nn.c, nn.rank, nn.c, nullptr, (int)nn.c0, tmp));
                    push_nn_chunks(B.nn, vnn(nn.V, nn.r, nn.rank, nn.r, Rj, 0, tmp, true));
                    pl->bytes += 2.0 * sizeof(T) * nn.rank * (nn.r + nn.c);
                }
            }
            emit(L_TN, o2, B.tn.size() - o2, 0);
            emit(L_NN, o3, B.nn.size() - o3, 0);
            ib_forward(l);
        }
        for (int l = S.nlevels - 1; l >= 0; --l) {
            ib_backward(l);
            size_t o2 = B.tn.size();
            size_t zi = 0;
            std::vector<NnTask> nnb;
            for (int j : S.level_nodes[l]) {
                const NodeRT& nn = nd[j];
                if (nn.r == 0) continue;
                const int32_t* Rj = d_rows + S.rows_ptr[j];
                if (!nn.compressed) {   // y_C -= L^O_j^T y_R
                    push_tn_chunks(B.tn, vtn(arena + nn.off + nn.c, nn.ld, nn.c, nn.r, Rj, 0, pl->y + nn.c0 * N, -1.0, 1.0));
                } else if (nn.rank) {   // y_C -= U_j (V_j^T y_R)
                    T* tmp = ztmp[l][zi++];
                    push_tn_chunks(B.tn, vtn(nn.V, nn.r, nn.rank, nn.r, Rj, 0, tmp));
                    push_nn_chunks(nnb, vnn(nn.U, nn.c, nn.rank, nn.c, nullptr, (int)nn.c0, tmp, false));
                }
            }
            emit(L_TN, o2, B.tn.size() - o2, 0);
            size_t o3 = B.nn.size();
            B.nn.insert(B.nn.end(), nnb.begin(), nnb.end());
            emit(L_NN, o3, nnb.size(), 0);
            std::vector<std::vector<Act>> acts;
            std::vector<int> big;
            std::vector<NnTask> hnn;
            size_t oh = B.tn.size();
            for (int j : S.level_nodes[l])
                if (nd[j].hier) hier_terms(j, true, B.tn, hnn);
            emit(L_TN, oh, B.tn.size() - oh, 0);
            size_t o = B.trsv.size();
            for (int j : S.level_nodes[l]) {
                const NodeRT& nn = nd[j];
                if (nn.hier) hier_leaves(j, true);
                else if (nn.c <= SOLVE_MAX) B.trsv.push_back(TrsvTask{inv_block(j, 0), nn.c, nn.c, N, pl->y + nn.c0 * N, N, 1});
                else big.push_back(j);
            }
            emit(L_TRSV, o, B.trsv.size() - o, 0);
            size_t ohn = B.nn.size();
            B.nn.insert(B.nn.end(), hnn.begin(), hnn.end());
            emit(L_NN, ohn, hnn.size(), 0);
            emit_hsolve(big, true, acts);
            emit_acts(acts);
        }
        emit(L_PERM_OUT, 0, 1, 0);
        if (zcur > pl->tmp + std::max<long long>(tmp_total, 1)) throw Error(RSC_ERR_CUDA, "solve scratch overflow");
        pl->hacts = pl->mem.upload(HA, stream);
        for (auto& h : HT) h.acts = pl->hacts + (intptr_t)h.acts;
        pl->hs = pl->mem.upload(HT, stream);
        pl->trsv = pl->mem.upload(B.trsv, stream);
        {   // long TN tasks: rows split over CTAs with per-task partial sums and arrival counters
            // (kept in the plan; each counter is back at zero when its launch ends)
            const int ych = N == 1 ? 1 : cdiv(N, 64), wcols = ap_tn_cols();
            auto split_of = [&](const TnTask& t) {
                if (N == 1) return t.nrow > TN1_SPLIT_ROWS ? cdiv(t.nrow, TN1_SPLIT_ROWS) : 1;
                return t.nrow >= TN_SPLIT_MIN ? std::min(cdiv(t.nrow, TN_SPLIT_ROWS), TN_SPLIT_MAX) : 1;
            };
            long long npart = 0, ncnt = 0;
            for (auto& t : B.tn) {
                const int ns = split_of(t);
                if (ns > 1) { npart += (long long)ns * wcols * N; ncnt += ych; }
            }
            T* part = npart ? (T*)pl->mem.alloc(sizeof(T) * npart) : nullptr;
            unsigned* cnt = ncnt ? (unsigned*)pl->mem.alloc(sizeof(unsigned) * ncnt) : nullptr;
            if (ncnt) CK(cudaMemsetAsync(cnt, 0, sizeof(unsigned) * ncnt, stream));
            for (auto& t : B.tn) {
                const int ns = split_of(t);
                if (ns == 1) continue;
                t.nsplit = ns;
                t.rps = cdiv(t.nrow, ns);
                t.part = part; part += (size_t)ns * wcols * N;
                t.cnt = cnt; cnt += ych;
            }
            for (Launch& L : pl->seq)
                if (L.kind == L_TN)
                    for (int i = 0; i < L.count; ++i) L.flag = std::max(L.flag, B.tn[L.off + i].nsplit);
        }
        pl->tn = pl->mem.upload(B.tn, stream);
        pl->nn = pl->mem.upload(B.nn, stream);
        if (!B.copy.empty()) pl->copy = pl->mem.upload(B.copy, stream);
        if (!B.csr.empty()) pl->csr = pl->mem.upload(B.csr, stream);
        for (auto& t : B.tn) pl->flops += 2.0 * t.nrow * std::min(ap_tn_cols(), t.K - t.t0) * N;
        for (auto& t : B.nn) pl->flops += 2.0 * std::min(NN_ROWS, t.nrow - t.row0) * t.K * N;
        pl->bytes += (4.0 * sizeof(T) * n + 16.0 * n) * N;
        sync_stream();
        // capture the launch list once
        CK(cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal));
        issue_apply(*pl, stream);
        cudaGraph_t g = nullptr;
        CK(cudaStreamEndCapture(stream, &g));
        CK(cudaGraphInstantiate(&pl->graph, g, 0));
        CK(cudaGraphDestroy(g));
        pl->mem.trim();
    }

    bool no_graph = std::getenv("RSC_NO_GRAPH") != nullptr;   // measurement aid: per-kernel apply profile
    void issue_apply(const ApplyPlan& A, cudaStream_t s, bool profiled = false) {
        const long long n = S.n;
        const int N = A.N;
        Profiler off;
        Profiler& P = profiled ? prof : off;
        const unsigned pg = (unsigned)std::min<long long>(cdiv(n, 256), 4096);
        for (const Launch& L : A.seq) {
            switch (L.kind) {
                case L_PERM_IN:
                    if (N == 1) PROF(P, "ap_perm", s, 0, 0, k_perm_in<T><<<pg, 256, 0, s>>>(A.gin, d_perm, A.y, n));
                    else PROF(P, "ap_perm", s, 0, 0, k_perm_in_cols<T><<<dim3(pg, N), 256, 0, s>>>(A.gin, d_perm, A.y, n, N));
                    break;
                case L_PERM_OUT:
                    if (N == 1) PROF(P, "ap_perm", s, 0, 0, k_perm_out<T><<<pg, 256, 0, s>>>(A.y, d_perm, A.gout, n));
                    else PROF(P, "ap_perm", s, 0, 0, k_perm_out_cols<T><<<dim3(pg, N), 256, 0, s>>>(A.y, d_perm, A.gout, n, N));
                    break;
                case L_TRSV:
                    if (N == 1) PROF(P, "ap_trsv", s, 0, 0, k_trsv<T, 1><<<L.count, 256, 0, s>>>(A.trsv + L.off));
                    else PROF(P, "ap_trsv", s, 0, 0,
                              k_trsv<T, TRSV_CW><<<dim3(L.count, cdiv(N, TRSV_CW)), 256, 0, s>>>(A.trsv + L.off));
                    break;
                case L_TN:
                    if (N == 1)
                        PROF(P, "ap_tn", s, 0, 0, k_tn1<T><<<dim3(L.count, 1, std::max(L.flag, 1)), 256, 0, s>>>(A.tn + L.off));
                    else {   // several right-hand sides: the staged kernel, 64 columns of A per CTA
                        const dim3 g((unsigned)L.count, (unsigned)cdiv(N, 64), (unsigned)std::max(L.flag, 1));
                        const int np = std::min(N, 64) <= 16 ? 16 : std::min(N, 64) <= 32 ? 32 : 64;
                        if (np == 16) PROF(P, "ap_tn", s, 0, 0, k_tn_s<T, 16><<<g, 256, ts_smem_bytes<T>(16), s>>>(A.tn + L.off));
                        else if (np == 32) PROF(P, "ap_tn", s, 0, 0, k_tn_s<T, 32><<<g, 256, ts_smem_bytes<T>(32), s>>>(A.tn + L.off));
                        else PROF(P, "ap_tn", s, 0, 0, k_tn_s<T, 64><<<g, 256, ts_smem_bytes<T>(64), s>>>(A.tn + L.off));
                    }
                    break;
                case L_NN:
                    PROF(P, "ap_nn", s, 0, 0, k_nn<T><<<dim3(L.count, cdiv(N, 16)), NN_ROWS, 0, s>>>(A.nn + L.off));
                    break;
                case L_COPY:
                    PROF(P, "ap_copy", s, 0, 0, k_copy<T><<<dim3(L.count, 32), 256, 0, s>>>(A.copy + L.off));
                    break;
                case L_CSR:
                    PROF(P, "ap_csr", s, 0, 0, k_csr_mm<T><<<dim3(L.count, cdiv(N, 16)), 256, 0, s>>>(A.csr + L.off));
                    break;
                case L_HSOLVE: {
                    const int cw = N == 1 ? 1 : std::max(1, std::min(pick_cw(L.flag), 8));
                    const dim3 g((unsigned)L.count, (unsigned)cdiv(N, cw));
                    switch (cw) {
                        case 8: PROF(P, "ap_hsolve", s, 0, 0, k_hsolve<T, 8><<<g, HS_THREADS, hs_smem(L.flag, 8), s>>>(A.hs + L.off)); break;
                        case 4: PROF(P, "ap_hsolve", s, 0, 0, k_hsolve<T, 4><<<g, HS_THREADS, hs_smem(L.flag, 4), s>>>(A.hs + L.off)); break;
                        case 2: PROF(P, "ap_hsolve", s, 0, 0, k_hsolve<T, 2><<<g, HS_THREADS, hs_smem(L.flag, 2), s>>>(A.hs + L.off)); break;
                        default: PROF(P, "ap_hsolve", s, 0, 0, k_hsolve<T, 1><<<g, HS_THREADS, hs_smem(L.flag, 1), s>>>(A.hs + L.off)); break;
                    }
                    break;
                }
            }
        }
        LAUNCH_CHECK();
    }

    void run_plan(const ApplyPlan& A, const double* d_r, double* d_z, cudaStream_t s) {
        const size_t bytes = sizeof(double) * S.n * A.N;
        if (d_r != A.gin) CK(cudaMemcpyAsync(A.gin, d_r, bytes, cudaMemcpyDeviceToDevice, s));
        if (no_graph) issue_apply(A, s, true);
        else PROF(prof, "apply", s, A.flops, A.bytes, CK(cudaGraphLaunch(A.graph, s)));
        launches += (long long)A.seq.size();
        if (d_z != A.gout) CK(cudaMemcpyAsync(d_z, A.gout, bytes, cudaMemcpyDeviceToDevice, s));
    }
    void apply(const double* d_r, double* d_z, cudaStream_t s) override {
        if (plan1.gen != factor_gen || !plan1.graph) {
            HostTimer ht_(this, "h_solve_plan");
            build_solve_plan(1);
        }
        run_plan(plan1, d_r, d_z, s);
    }
    long long n_of() const override { return S.n; }
    // nrhs right-hand sides at once (column c at d_r + c n): one pass over the factor for all
    void prepare_multi(int nrhs) override {
        if (nrhs > 1 && (planN.N != nrhs || planN.gen != factor_gen || !planN.graph)) {
            HostTimer ht_(this, "h_solve_plan");
            build_solve_plan(nrhs);
            pl = &plan1;
        }
    }
    void apply_multi(const double* d_r, double* d_z, int nrhs, cudaStream_t s) override {
        if (nrhs == 1) { apply(d_r, d_z, s); return; }
        prepare_multi(nrhs);
        run_plan(planN, d_r, d_z, s);
    }

    // ---------------------------------------------------------------- allocation-free apply
    // The same level-by-level launch list as build_solve_plan (persistent solves for
    // hierarchical and large dense blocks), but every buffer it needs -- the permuted
    // work vector, the low-rank temporaries and the task records -- lives in the
    // caller-provided static device region `base` (cap bytes).  Loading the records
    // copies host-built vectors into that region on the caller's stream; nothing is
    // allocated on the device.
    long long factor_gen = 0;
    long long generation() const override { return factor_gen; }
    std::vector<Launch> na_seq;
    T* na_y = nullptr;
    const TrsvTask* na_trsv = nullptr;
    const TnTask* na_tn = nullptr;
    const NnTask* na_nn = nullptr;
    const HTask* na_hs = nullptr;

    rsc_status load_noalloc(char* base, size_t cap, cudaStream_t s) {
        if (ib_on) throw Error(RSC_ERR_INVALID_ARG, "the allocation-free apply does not take interior blocks");
        auto align = [](size_t x) { return (x + 255) / 256 * 256; };
        const long long n = S.n;
        long long tmp_total = 0;
        for (int j = 0; j < S.M; ++j) tmp_total += nd[j].compressed ? nd[j].rank : 0;
        size_t off = 0;
        T* y = (T*)(base + off);
        off = align(off + sizeof(T) * n);
        T* tmp = (T*)(base + off);
        off = align(off + sizeof(T) * std::max<long long>(tmp_total, 1));
        if (off > cap)
            throw Error(RSC_ERR_INVALID_ARG, "problem needs " + std::to_string(off) +
                                                 " bytes of static scratch for its vectors; the library holds " +
                                                 std::to_string(cap));
        std::vector<HAct> HA;
        std::vector<HTask> HT;
        std::vector<TrsvTask> TV;
        std::vector<TnTask> TN;
        std::vector<NnTask> NN;
        std::vector<Launch> q;
        T* zc = tmp;
        auto emit = [&](int kind, size_t o, size_t cnt, int flag) {
            if (cnt) q.push_back(Launch{kind, (int)cnt, o, flag});
        };
        auto tn_chunks = [&](const TnTask& t) {
            for (int t0 = 0; t0 < t.K; t0 += TN_COLS) { TnTask c = t; c.t0 = t0; TN.push_back(c); }
        };
        auto nn_chunks = [&](const NnTask& t, std::vector<NnTask>& dst) {
            for (int r0 = 0; r0 < t.nrow; r0 += NN_ROWS) { NnTask c = t; c.row0 = r0; dst.push_back(c); }
        };
        auto hsolve = [&](const std::vector<int>& nodes, bool tr) {
            const size_t o = HT.size();
            int maxc = 0;
            for (int j : nodes) {
                if (pick_cw(nd[j].c) == 0)
                    throw Error(RSC_ERR_INVALID_ARG, "a diagonal block is too large for the allocation-free apply");
                const long long first = (long long)HA.size();
                const double keep = flops;
                hacts(j, 0, tr, HA);
                flops = keep;
                HT.push_back(HTask{(const HAct*)(intptr_t)first, (long long)HA.size() - first, y + nd[j].c0, 1, 1,
                                   nd[j].c, tr ? 1 : 0});
                maxc = std::max(maxc, nd[j].c);
            }
            emit(L_HSOLVE, o, HT.size() - o, maxc);
        };
        std::vector<std::vector<T*>> zt(S.nlevels);
        for (int l = 0; l < S.nlevels; ++l) {
            size_t o = TV.size();
            std::vector<int> big;
            for (int j : S.level_nodes[l]) {
                const NodeRT& nn = nd[j];
                if (!nn.hier && nn.c <= SOLVE_MAX) TV.push_back(TrsvTask{inv_block(j, 0), nn.c, nn.c, 1, y + nn.c0, 1, 0});
                else big.push_back(j);
            }
            emit(L_TRSV, o, TV.size() - o, 0);
            hsolve(big, false);
            const size_t o2 = TN.size(), o3 = NN.size();
            for (int j : S.level_nodes[l]) {
                const NodeRT& nn = nd[j];
                if (nn.r == 0) continue;
                const int32_t* Rj = d_rows + S.rows_ptr[j];
                if (!nn.compressed) {
                    nn_chunks(nn_task(arena + nn.off + nn.c, nn.ld, nn.c, nn.r, nullptr, 0, Rj, 0, y + nn.c0, 1, y, 1, 1,
                                      -1.0, true), NN);
                } else if (nn.rank) {
                    T* t = zc;
                    zc += nn.rank;
                    zt[l].push_back(t);
                    tn_chunks(tn_task(nn.U, nn.c, nn.rank, nn.c, nullptr, 0, nullptr, (int)nn.c0, y, 1, t, 1, 1));
                    nn_chunks(nn_task(nn.V, nn.r, nn.rank, nn.r, nullptr, 0, Rj, 0, t, 1, y, 1, 1, -1.0, true), NN);
                }
            }
            emit(L_TN, o2, TN.size() - o2, 0);
            emit(L_NN, o3, NN.size() - o3, 0);
        }
        for (int l = S.nlevels - 1; l >= 0; --l) {
            const size_t o2 = TN.size();
            size_t zi = 0;
            std::vector<NnTask> nb;
            for (int j : S.level_nodes[l]) {
                const NodeRT& nn = nd[j];
                if (nn.r == 0) continue;
                const int32_t* Rj = d_rows + S.rows_ptr[j];
                if (!nn.compressed) {
                    tn_chunks(tn_task(arena + nn.off + nn.c, nn.ld, nn.c, nn.r, nullptr, 0, Rj, 0, y, 1, y + nn.c0, 1, 1,
                                      -1.0, 1.0));
                } else if (nn.rank) {
                    T* t = zt[l][zi++];
                    tn_chunks(tn_task(nn.V, nn.r, nn.rank, nn.r, nullptr, 0, Rj, 0, y, 1, t, 1, 1));
                    nn_chunks(nn_task(nn.U, nn.c, nn.rank, nn.c, nullptr, 0, nullptr, (int)nn.c0, t, 1, y, 1, 1, -1.0,
                                      false), nb);
                }
            }
            emit(L_TN, o2, TN.size() - o2, 0);
            const size_t o3 = NN.size();
            NN.insert(NN.end(), nb.begin(), nb.end());
            emit(L_NN, o3, nb.size(), 0);
            std::vector<int> big;
            for (int j : S.level_nodes[l])
                if (nd[j].hier || nd[j].c > SOLVE_MAX) big.push_back(j);
            hsolve(big, true);
            const size_t o = TV.size();
            for (int j : S.level_nodes[l]) {
                const NodeRT& nn = nd[j];
                if (!nn.hier && nn.c <= SOLVE_MAX) TV.push_back(TrsvTask{inv_block(j, 0), nn.c, nn.c, 1, y + nn.c0, 1, 1});
            }
            emit(L_TRSV, o, TV.size() - o, 0);
        }
        const size_t ha = off; off = align(off + sizeof(HAct) * HA.size());
        const size_t hs = off; off = align(off + sizeof(HTask) * HT.size());
        const size_t tv = off; off = align(off + sizeof(TrsvTask) * TV.size());
        const size_t tn = off; off = align(off + sizeof(TnTask) * TN.size());
        const size_t nnq = off; off = align(off + sizeof(NnTask) * NN.size());
        if (off > cap)
            throw Error(RSC_ERR_INVALID_ARG, "problem needs " + std::to_string(off) +
                                                 " bytes of static scratch; the library holds " + std::to_string(cap));
        for (auto& h : HT) h.acts = (const HAct*)(base + ha) + (intptr_t)h.acts;
        auto put = [&](size_t o, const void* src, size_t bytes) {
            if (bytes) CK(cudaMemcpyAsync(base + o, src, bytes, cudaMemcpyHostToDevice, s));
        };
        put(ha, HA.data(), sizeof(HAct) * HA.size());
        put(hs, HT.data(), sizeof(HTask) * HT.size());
        put(tv, TV.data(), sizeof(TrsvTask) * TV.size());
        put(tn, TN.data(), sizeof(TnTask) * TN.size());
        put(nnq, NN.data(), sizeof(NnTask) * NN.size());
        na_seq = std::move(q);
        na_y = y;
        na_hs = (const HTask*)(base + hs);
        na_trsv = (const TrsvTask*)(base + tv);
        na_tn = (const TnTask*)(base + tn);
        na_nn = (const NnTask*)(base + nnq);
        return RSC_OK;
    }

    long long na_loaded_gen = -1;
    bool noalloc_ready() const override { return na_y != nullptr && na_loaded_gen == factor_gen; }
    rsc_status apply_noalloc(const double* d_r, double* d_z, cudaStream_t s, char* base, size_t cap,
                             bool load) override {
        if (load) {
            na_y = nullptr;
            load_noalloc(base, cap, s);
            na_loaded_gen = factor_gen;
        }
        const long long n = S.n;
        k_perm_in<T><<<std::min(cdiv(n, 256), 4096), 256, 0, s>>>(d_r, d_perm, na_y, n);
        for (const Launch& L : na_seq) {
            switch (L.kind) {
                case L_TRSV: k_trsv<T, 1><<<L.count, 256, 0, s>>>(na_trsv + L.off); break;
                case L_TN: k_tn1<T><<<L.count, 256, 0, s>>>(na_tn + L.off); break;
                case L_NN: k_nn<T><<<L.count, NN_ROWS, 0, s>>>(na_nn + L.off); break;
                case L_HSOLVE: k_hsolve<T, 1><<<L.count, HS_THREADS, hs_smem(L.flag, 1), s>>>(na_hs + L.off); break;
                default: break;
            }
        }
        k_perm_out<T><<<std::min(cdiv(n, 256), 4096), 256, 0, s>>>(na_y, d_perm, d_z, n);
        LAUNCH_CHECK();
        return RSC_OK;
    }

    // ---------------------------------------------------------------- introspection
    void node_info(int j, int32_t* info) const override {
        const NodeRT& n = nd[j];
        info[2] = n.compressed ? 1 : 0;
        info[3] = n.rank;
        info[4] = n.hier ? 1 : 0;
        info[5] = n.hier ? S.tree[j].nblocks : 1;
    }

    template <class X> std::vector<X> dl(const X* p, size_t cnt) const {
        std::vector<X> v(cnt);
        if (cnt) CK(cudaMemcpy(v.data(), p, sizeof(X) * cnt, cudaMemcpyDeviceToHost));
        return v;
    }

    rsc_status node_blocks(int j, double* LD, double* LO) override {
        CK(cudaStreamSynchronize(stream));
        const NodeRT& n = nd[j];
        const int c = n.c, r = n.r;
        if (LD) {
            std::fill(LD, LD + (size_t)c * c, 0.0);
            if (!n.hier) {
                auto P = dl(arena + n.off, (size_t)n.ld * c);
                for (int q = 0; q < c; ++q)
                    for (int i = q; i < c; ++i) LD[i + (size_t)q * c] = (double)P[i + (size_t)q * n.ld];
            } else {
                const BlockTree& t = S.tree[j];
                for (int s = 1; s <= t.nblocks; ++s) {
                    if (t.leaf[s]) {
                        const int sz = t.hi[s] - t.lo[s];
                        auto P = dl(arena + n.leaf_off[s], (size_t)sz * sz);
                        for (int q = 0; q < sz; ++q)
                            for (int i = q; i < sz; ++i)
                                LD[(t.lo[s] + i) + (size_t)(t.lo[s] + q) * c] = (double)P[i + (size_t)q * sz];
                    } else if (n.brank[s]) {
                        const int rs = t.hi[s] - t.mid[s], cs = t.mid[s] - t.lo[s], q = n.brank[s];
                        auto V = dl(n.bV[s], (size_t)rs * q);
                        auto U = dl(n.bU[s], (size_t)cs * q);
                        for (int b = 0; b < cs; ++b)
                            for (int a = 0; a < rs; ++a) {
                                double v = 0.0;
                                for (int l = 0; l < q; ++l) v += (double)V[a + (size_t)l * rs] * (double)U[b + (size_t)l * cs];
                                LD[(t.mid[s] + a) + (size_t)(t.lo[s] + b) * c] = v;
                            }
                    }
                }
            }
        }
        const int rfull = S.nrows(j);
        if (LO && rfull > 0) {
            if (!n.compressed) {   // interior blocks: the rows after C_B are not stored (NaN)
                auto P = dl(arena + n.off, (size_t)n.ld * c);
                for (int q = 0; q < c; ++q)
                    for (int i = 0; i < rfull; ++i)
                        LO[i + (size_t)q * rfull] = i < r ? (double)P[c + i + (size_t)q * n.ld] : std::nan("");
            } else {
                std::fill(LO, LO + (size_t)r * c, 0.0);
                if (n.rank) {
                    auto V = dl(n.V, (size_t)r * n.rank);
                    auto U = dl(n.U, (size_t)c * n.rank);
                    for (int q = 0; q < c; ++q)
                        for (int i = 0; i < r; ++i) {
                            double v = 0.0;
                            for (int l = 0; l < n.rank; ++l) v += (double)V[i + (size_t)l * r] * (double)U[q + (size_t)l * c];
                            LO[i + (size_t)q * r] = v;
                        }
                }
            }
        }
        return RSC_OK;
    }

    void stats(rsc_stats_t* out) const override {
        double bytes = 0.0;
        int ncomp = 0, maxr = 0;
        for (int j = 0; j < S.M; ++j) {
            const NodeRT& n = nd[j];
            if (!n.compressed) bytes += (double)(n.c * (n.c + 1) / 2 + (double)n.r * n.c);
            else {
                ++ncomp;
                maxr = std::max(maxr, n.rank);
                bytes += (double)n.rank * (n.c + n.r);
                if (!n.hier) bytes += (double)n.c * (n.c + 1) / 2;
                else {
                    const BlockTree& t = S.tree[j];
                    for (int s = 1; s <= t.nblocks; ++s) {
                        if (t.leaf[s]) { double sz = t.hi[s] - t.lo[s]; bytes += sz * (sz + 1) / 2; }
                        else bytes += (double)n.brank[s] * (t.hi[s] - t.lo[s]);
                    }
                }
            }
        }
        out->factor_bytes = bytes * sizeof(T);
        out->factor_flops = flops;
        out->factor_seconds = factor_seconds;
        out->solve_seconds = solve_seconds;
        out->restarts = restarts;
        out->n_compressed = ncomp;
        out->max_rank = maxr;
        out->last_iters = last_iters;
        out->last_relres = last_relres;
        out->gpu_launches = launches;
    }
};

template <class T>
__global__ void k_strided_copy(const T* __restrict__ src, long long ssr, long long ssc, T* __restrict__ dst,
                               long long dsr, long long dsc, int m, int nc) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)m * nc;
         e += (long long)gridDim.x * blockDim.x) {
        long long i = e % m, c = e / m;
        dst[i * dsr + c * dsc] = src[i * ssr + c * ssc];
    }
}

// ------------------------------------------------------------------ static scratch of the allocation-free apply
// A fixed device region for rsc_apply_preconditioner_device_noalloc: every GPU that
// loads this library holds these 64 MiB until the process exits.  Host code must not
// use the symbol as an address: its device address is looked up once per device with
// cudaGetSymbolAddress (with that device current) and passed to the kernels.
constexpr size_t NOALLOC_SCRATCH_BYTES = (size_t)64 << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

namespace {
std::mutex g_na_mu;
std::map<int, char*> g_na_addr;                                   // device -> address of the region
std::map<int, std::pair<long long, long long>> g_na_loaded;       // device -> (engine uid, factor generation)
std::atomic<long long> g_engine_uid{0};
}  // namespace

// ------------------------------------------------------------------ Engine facade
Engine::Engine(const Symbolic& S, const rsc_options& o) {
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev == 0) throw Error(RSC_ERR_CUDA, "no CUDA device available");
    if (o.precision == RSC_PREC_FP64) impl_.reset(new EngineT<double>(S, o));
    else impl_.reset(new EngineT<float>(S, o));
    impl_->uid = ++g_engine_uid;
    CK(cudaGetDevice(&impl_->device));
}
Engine::~Engine() = default;
rsc_status Engine::factor(const double* val, double tol, const FixedRank* fr) { return impl_->factor(val, tol, fr); }

int rank_heuristic(int m, int n, double alpha, int p) {
    const int k = std::min(m, n);
    if (k <= 0) return 0;
    const double r = std::ceil(alpha * std::sqrt((double)k) * std::log2((double)k));
    return (int)std::min<double>(k, r + p);
}
void Engine::values_changed() {
    impl_->a_uploaded = false;
    impl_->vals_dev = false;   // the host copy holds the values again
}
rsc_status Engine::values_device(const double* d_val, long long nnz, void* stream) {
    impl_->set_values_device(d_val, nnz, stream ? (cudaStream_t)stream : impl_->stream);
    return RSC_OK;
}
bool Engine::factored() const { return impl_->factored(); }
rsc_status Engine::solve_host(const std::vector<int64_t>& rp, const std::vector<int32_t>& ci,
                              const std::vector<double>& val, const double* b, double* x, double rtol,
                              int32_t max_iter, int32_t* iters, double* relres) {
    const long long n = (long long)rp.size() - 1;
    cudaStream_t s = impl_->stream;
    double* d = nullptr;
    CK(cudaMalloc(&d, sizeof(double) * 2 * n));
    rsc_status st;
    try {
        CK(cudaMemcpyAsync(d, b, sizeof(double) * n, cudaMemcpyHostToDevice, s));
        st = impl_->pcg(rp, ci, val, d, d + n, rtol, max_iter, iters, relres, s);
        CK(cudaMemcpyAsync(x, d + n, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    } catch (...) {
        cudaFree(d);
        throw;
    }
    cudaFree(d);
    return st;
}
rsc_status Engine::solve_device(const std::vector<int64_t>& rp, const std::vector<int32_t>& ci,
                                const std::vector<double>& val, const double* d_b, double* d_x, double rtol,
                                int32_t max_iter, int32_t* iters, double* relres, void* stream) {
    cudaStream_t s = stream ? (cudaStream_t)stream : impl_->stream;
    rsc_status st = impl_->pcg(rp, ci, val, d_b, d_x, rtol, max_iter, iters, relres, s);
    CK(cudaStreamSynchronize(s));
    return st;
}
rsc_status Engine::solve_batch_device(const std::vector<int64_t>& rp, const std::vector<int32_t>& ci,
                                      const std::vector<double>& val, const std::vector<long long>& seg_ptr,
                                      const double* d_B, double* d_X, int nrhs, double rtol, int max_iter, int* iters,
                                      double* relres, void* stream) {
    cudaStream_t s = stream ? (cudaStream_t)stream : impl_->stream;
    rsc_status st = impl_->pcg_batch(rp, ci, val, seg_ptr, d_B, d_X, nrhs, rtol, max_iter, iters, relres, s);
    CK(cudaStreamSynchronize(s));
    return st;
}

rsc_status Engine::pattern_outer(const std::vector<int64_t>& rp, const std::vector<int32_t>& ci,
                                 const std::vector<double>& val, const double* d_u, const double* d_v, double alpha,
                                 double* d_out, void* stream) {
    cudaStream_t s = stream ? (cudaStream_t)stream : impl_->stream;
    impl_->pattern_outer(rp, ci, val, d_u, d_v, alpha, d_out, s);
    CK(cudaStreamSynchronize(s));
    return RSC_OK;
}

rsc_status Engine::apply_precond_noalloc(const double* d_r, double* d_z, void* stream) {
    cudaStream_t s = stream ? (cudaStream_t)stream : impl_->stream;
    // the records hold device addresses of the engine's device: the static region of another
    // device must never be paired with them
    int dev = 0;
    CK(cudaGetDevice(&dev));
    if (dev != impl_->device)
        throw Error(RSC_ERR_STATE, "the current CUDA device (" + std::to_string(dev) +
                                       ") is not the device the handle was factored on (" +
                                       std::to_string(impl_->device) + ")");
    std::lock_guard<std::mutex> lock(g_na_mu);
    auto it = g_na_addr.find(dev);
    if (it == g_na_addr.end()) {
        char* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress((void**)&p, g_noalloc_scratch);
        if (e != cudaSuccess) throw Error(RSC_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        it = g_na_addr.emplace(dev, p).first;
    }
    // reload when the region holds another engine's records or those of an earlier factor
    const std::pair<long long, long long> mine{impl_->uid, impl_->generation()};
    auto ld = g_na_loaded.find(dev);
    const bool load = ld == g_na_loaded.end() || ld->second != mine || !impl_->noalloc_ready();
    if (load) g_na_loaded.erase(dev);
    rsc_status st = impl_->apply_noalloc(d_r, d_z, s, it->second, NOALLOC_SCRATCH_BYTES, load);
    if (load) g_na_loaded[dev] = mine;
    CK(cudaStreamSynchronize(s));   // every call returns with its result in d_z
    return st;
}

rsc_status Engine::apply_precond(const double* d_r, double* d_z, void* stream) {
    cudaStream_t s = stream ? (cudaStream_t)stream : impl_->stream;
    impl_->apply(d_r, d_z, s);
    CK(cudaStreamSynchronize(s));
    return RSC_OK;
}
void Engine::node_info(int j, int32_t* info) const { impl_->node_info(j, info); }
rsc_status Engine::node_blocks(int j, double* LD, double* LO) const { return impl_->node_blocks(j, LD, LO); }
void Engine::stats(rsc_stats_t* out) const { impl_->stats(out); }
void Engine::profile(int enable, const char* only) {
    impl_->prof.flush();
    impl_->prof.acc.clear();
    impl_->prof.on = enable != 0;
    impl_->prof.only = only ? only : "";
}
std::string Engine::profile_json() { return impl_->prof.json(); }
std::string Engine::tuning_json() const { return impl_->tuner.json(); }
void Engine::set_wait_limit(long long polls) { impl_->rf_spin_limit = polls > 0 ? (unsigned long long)polls : RFP_SPIN_LIMIT; }

}  // namespace rsc
