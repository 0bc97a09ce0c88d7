// GPU engine: device memory, the factorization driver and the PCG solve.
#pragma once

#include <cstdint>
#include <memory>
#include <stdexcept>
#include <string>
#include <vector>

#include "rsc.h"
#include "rsc_internal.h"

namespace rsc {

struct Error : std::runtime_error {
    rsc_status status;
    Error(rsc_status s, const std::string& m) : std::runtime_error(m), status(s) {}
};

struct EngineImpl;

// Section 5.2's fixed-rank form of Alg. 3: block B (m x n) gets the rank of Eq. rankFunction,
// ceil(alpha sqrt(k) log2 k) + p with k = min(m, n), capped at k; alpha_O for off-diagonal
// blocks, alpha_D (grown by 1.25 per indefinite restart, Section 5.3) for diagonal blocks.
struct FixedRank {
    double alpha_O = 0.0, alpha_D = 0.0;
    int p = 0;
};
int rank_heuristic(int m, int n, double alpha, int p);

class Engine {
public:
    Engine(const Symbolic& S, const rsc_options& o);
    ~Engine();
    rsc_status factor(const double* val, double tol, const FixedRank* fr = nullptr);
    void values_changed();   // new values of A: the SpMV copy is refreshed by the next solve
    rsc_status values_device(const double* d_val, long long nnz, void* stream);   // new values, on the device
    bool factored() const;
    rsc_status solve_host(const std::vector<int64_t>& rp, const std::vector<int32_t>& ci,
                          const std::vector<double>& val, const double* b, double* x, double rtol,
                          int32_t max_iter, int32_t* iters, double* relres);
    rsc_status solve_device(const std::vector<int64_t>& rp, const std::vector<int32_t>& ci,
                            const std::vector<double>& val, const double* d_b, double* d_x, double rtol,
                            int32_t max_iter, int32_t* iters, double* relres, void* stream);
    rsc_status apply_precond(const double* d_r, double* d_z, void* stream);
    rsc_status apply_precond_noalloc(const double* d_r, double* d_z, void* stream);
    rsc_status solve_batch_device(const std::vector<int64_t>& rp, const std::vector<int32_t>& ci,
                                  const std::vector<double>& val, const std::vector<long long>& seg_ptr,
                                  const double* d_B, double* d_X, int nrhs, double rtol, int max_iter, int* iters,
                                  double* relres, void* stream);
    rsc_status pattern_outer(const std::vector<int64_t>& rp, const std::vector<int32_t>& ci,
                             const std::vector<double>& val, const double* d_u, const double* d_v, double alpha,
                             double* d_out, void* stream);
    void node_info(int j, int32_t* info) const;
    rsc_status node_blocks(int j, double* LD, double* LO) const;
    void stats(rsc_stats_t* out) const;
    void profile(int enable, const char* only);
    std::string profile_json();
    std::string tuning_json() const;
    void set_wait_limit(long long polls);

private:
    std::unique_ptr<EngineImpl> impl_;
};

}  // namespace rsc
