// C ABI entry points (include/rsc.h).  Argument checking, error capture and
// dispatch into the host symbolic analysis and the GPU engine.
#include <cmath>
#include <cstring>
#include <exception>
#include <new>
#include <string>

#include "engine.h"
#include "rsc_internal.h"

using rsc::Engine;
using rsc::FixedRank;

struct rsc_handle {
    rsc::Symbolic sym;
    rsc_options opts;
    std::vector<double> val;      // caller's values (original order)
    std::vector<int64_t> row_ptr; // caller's pattern (original order)
    std::vector<int32_t> col_idx;
    Engine* eng = nullptr;
    std::string err;
};

namespace {
thread_local std::string g_last_error;

rsc_status fail(rsc_handle* h, rsc_status s, const std::string& msg) {
    if (h) h->err = msg;
    g_last_error = msg;
    return s;
}

template <class F>
rsc_status guarded(rsc_handle* h, F&& f) {
    try {
        return f();
    } catch (const std::bad_alloc&) {
        return fail(h, RSC_ERR_OOM, "host allocation failed");
    } catch (const rsc::Error& e) {
        return fail(h, e.status, e.what());
    } catch (const std::exception& e) {
        return fail(h, RSC_ERR_CUDA, e.what());
    } catch (...) {
        return fail(h, RSC_ERR_CUDA, "unknown error");
    }
}
}  // namespace

extern "C" {

rsc_status rsc_options_default(rsc_options* o) {
    if (!o) return RSC_ERR_INVALID_ARG;
    std::memset(o, 0, sizeof(*o));
    o->tau_O = 256;
    o->tau_D = 256;
    o->leaf_size = 64;
    o->sample_block = 16;
    o->power_iters = 0;
    o->dof_per_node = 1;
    o->max_restarts = 8;
    o->precision = RSC_PREC_FP64;
    o->diag_compress = 1;
    o->seed = 0;
    o->amalgamate = 0;
    o->interior_blocks = 0;
    return RSC_OK;
}

rsc_status rsc_analyze(int64_t n, const int64_t* row_ptr, const int32_t* col_idx, const double* val,
                       const double* coords, const rsc_options* opts, rsc_handle** out) {
    if (!out) return fail(nullptr, RSC_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    rsc_handle* h = nullptr;
    rsc_status st = guarded(nullptr, [&]() -> rsc_status {
        rsc_options o;
        if (opts) o = *opts; else rsc_options_default(&o);
        if (o.precision < RSC_PREC_FP64 || o.precision > RSC_PREC_BF16)
            return fail(nullptr, RSC_ERR_INVALID_ARG, "unknown precision");
        if (o.power_iters < 0 || o.max_restarts < 0)
            return fail(nullptr, RSC_ERR_INVALID_ARG, "power_iters and max_restarts must be >= 0");
        if (o.amalgamate != 0 && o.amalgamate != 1)
            return fail(nullptr, RSC_ERR_INVALID_ARG, "amalgamate must be 0 or 1");
        if (o.interior_blocks != 0 && o.interior_blocks != 1)
            return fail(nullptr, RSC_ERR_INVALID_ARG, "interior_blocks must be 0 or 1");
        h = new rsc_handle();
        h->opts = o;
        std::string why = rsc::analyze_symbolic(n, row_ptr, col_idx, val, coords, o, h->sym);
        if (!why.empty()) {
            delete h;
            h = nullptr;
            return fail(nullptr, RSC_ERR_INVALID_ARG, why);
        }
        h->val.assign(val, val + row_ptr[n]);
        h->row_ptr.assign(row_ptr, row_ptr + n + 1);
        h->col_idx.assign(col_idx, col_idx + row_ptr[n]);
        return RSC_OK;
    });
    if (st == RSC_OK) *out = h;
    else delete h;
    return st;
}

rsc_status rsc_get_ordering(const rsc_handle* h, int32_t* perm, int32_t* n_snodes, int64_t* snode_ptr) {
    if (!h) return fail(nullptr, RSC_ERR_INVALID_ARG, "NULL handle");
    const auto& S = h->sym;
    if (perm) std::memcpy(perm, S.perm.data(), sizeof(int32_t) * S.n);
    if (n_snodes) *n_snodes = S.M;
    if (snode_ptr) std::memcpy(snode_ptr, S.sn_ptr.data(), sizeof(int64_t) * (S.M + 1));
    return RSC_OK;
}

rsc_status rsc_get_coordinates(const rsc_handle* h, double* pos) {
    if (!h || !pos) return fail(nullptr, RSC_ERR_INVALID_ARG, "NULL handle or pos");
    std::memcpy(pos, h->sym.node_pos.data(), sizeof(double) * h->sym.node_pos.size());
    return RSC_OK;
}

rsc_status rsc_get_structure(const rsc_handle* h, int64_t* rows_ptr, int32_t* rows, int32_t* parent,
                             int32_t* level, int32_t* kind) {
    if (!h) return fail(nullptr, RSC_ERR_INVALID_ARG, "NULL handle");
    const auto& S = h->sym;
    if (rows_ptr) std::memcpy(rows_ptr, S.rows_ptr.data(), sizeof(int64_t) * (S.M + 1));
    if (rows) std::memcpy(rows, S.rows.data(), sizeof(int32_t) * S.rows.size());
    if (parent) std::memcpy(parent, S.parent.data(), sizeof(int32_t) * S.M);
    if (level) std::memcpy(level, S.level.data(), sizeof(int32_t) * S.M);
    if (kind)
        for (int j = 0; j < S.M; ++j) kind[j] = S.kind[j];
    return RSC_OK;
}

rsc_status rsc_factor(rsc_handle* h, double tol) {
    if (!h) return fail(nullptr, RSC_ERR_INVALID_ARG, "NULL handle");
    return guarded(h, [&]() -> rsc_status {
        if (!h->eng) h->eng = new Engine(h->sym, h->opts);
        return h->eng->factor(h->val.data(), tol);
    });
}

rsc_status rsc_factor_fixed_rank(rsc_handle* h, double alpha_O, double alpha_D, int32_t p) {
    if (!h) return fail(nullptr, RSC_ERR_INVALID_ARG, "NULL handle");
    if (!(std::isfinite(alpha_O) && alpha_O >= 0) || !(std::isfinite(alpha_D) && alpha_D >= 0) || p < 0)
        return fail(h, RSC_ERR_INVALID_ARG, "alpha_O, alpha_D and p must be finite and >= 0");
    return guarded(h, [&]() -> rsc_status {
        if (!h->eng) h->eng = new Engine(h->sym, h->opts);
        FixedRank fr;
        fr.alpha_O = alpha_O;
        fr.alpha_D = alpha_D;
        fr.p = p;
        return h->eng->factor(h->val.data(), 0.0, &fr);
    });
}

rsc_status rsc_refactor_values(rsc_handle* h, const double* val) {
    if (!h) return fail(nullptr, RSC_ERR_INVALID_ARG, "NULL handle");
    if (!val) return fail(h, RSC_ERR_INVALID_ARG, "val is NULL");
    for (size_t e = 0; e < h->val.size(); ++e)
        if (!std::isfinite(val[e])) return fail(h, RSC_ERR_INVALID_ARG, "non-finite matrix value");
    std::memcpy(h->val.data(), val, sizeof(double) * h->val.size());
    if (h->eng) h->eng->values_changed();
    return RSC_OK;
}

rsc_status rsc_refactor_values_device(rsc_handle* h, const double* d_val, void* stream) {
    if (!h) return fail(nullptr, RSC_ERR_INVALID_ARG, "NULL handle");
    if (!d_val) return fail(h, RSC_ERR_INVALID_ARG, "d_val is NULL");
    return guarded(h, [&]() -> rsc_status {
        if (!h->eng) h->eng = new Engine(h->sym, h->opts);
        return h->eng->values_device(d_val, (long long)h->val.size(), stream);
    });
}

rsc_status rsc_solve(rsc_handle* h, const double* b, double* x, double rtol, int32_t max_iter, int32_t* iters,
                     double* final_relres) {
    if (!h) return fail(nullptr, RSC_ERR_INVALID_ARG, "NULL handle");
    if (!b || !x) return fail(h, RSC_ERR_INVALID_ARG, "b and x are required");
    return guarded(h, [&]() -> rsc_status {
        if (!h->eng || !h->eng->factored()) return fail(h, RSC_ERR_STATE, "rsc_solve before rsc_factor");
        return h->eng->solve_host(h->row_ptr, h->col_idx, h->val, b, x, rtol, max_iter, iters, final_relres);
    });
}

rsc_status rsc_solve_device(rsc_handle* h, const double* d_b, double* d_x, double rtol, int32_t max_iter,
                            int32_t* iters, double* final_relres, void* stream) {
    if (!h) return fail(nullptr, RSC_ERR_INVALID_ARG, "NULL handle");
    if (!d_b || !d_x) return fail(h, RSC_ERR_INVALID_ARG, "d_b and d_x are required");
    return guarded(h, [&]() -> rsc_status {
        if (!h->eng || !h->eng->factored()) return fail(h, RSC_ERR_STATE, "rsc_solve_device before rsc_factor");
        return h->eng->solve_device(h->row_ptr, h->col_idx, h->val, d_b, d_x, rtol, max_iter, iters,
                                    final_relres, stream);
    });
}

rsc_status rsc_apply_preconditioner_device(rsc_handle* h, const double* d_r, double* d_z, void* stream) {
    if (!h) return fail(nullptr, RSC_ERR_INVALID_ARG, "NULL handle");
    if (!d_r || !d_z) return fail(h, RSC_ERR_INVALID_ARG, "d_r and d_z are required");
    return guarded(h, [&]() -> rsc_status {
        if (!h->eng || !h->eng->factored()) return fail(h, RSC_ERR_STATE, "apply before rsc_factor");
        return h->eng->apply_precond(d_r, d_z, stream);
    });
}

rsc_status rsc_apply_preconditioner_device_noalloc(rsc_handle* h, const double* d_r, double* d_z, void* stream) {
    if (!h) return fail(nullptr, RSC_ERR_INVALID_ARG, "NULL handle");
    if (!d_r || !d_z) return fail(h, RSC_ERR_INVALID_ARG, "d_r and d_z are required");
    return guarded(h, [&]() -> rsc_status {
        if (!h->eng || !h->eng->factored()) return fail(h, RSC_ERR_STATE, "apply before rsc_factor");
        return h->eng->apply_precond_noalloc(d_r, d_z, stream);
    });
}

// independent systems = connected components; each must be a contiguous row range
static bool system_ranges(const rsc::Symbolic& S, std::vector<long long>& seg) {
    const int dof = S.dof;
    const int64_t nodes = S.n / dof;
    seg.assign(1, 0);
    // components are numbered by their smallest node: contiguous ranges step by one
    for (int64_t v = 1; v < nodes; ++v)
        if (S.comp_of[v] != S.comp_of[v - 1]) {
            if (S.comp_of[v] != S.comp_of[v - 1] + 1) return false;
            seg.push_back(v * dof);
        }
    seg.push_back(S.n);
    return (int)seg.size() - 1 == S.ncomp;
}

rsc_status rsc_get_systems(const rsc_handle* h, int32_t* n_systems, int64_t* sys_ptr) {
    if (!h || !n_systems) return fail(nullptr, RSC_ERR_INVALID_ARG, "NULL argument");
    std::vector<long long> seg;
    if (!system_ranges(h->sym, seg))
        return fail(const_cast<rsc_handle*>(h), RSC_ERR_INVALID_ARG,
                    "independent systems do not occupy contiguous row ranges");
    *n_systems = (int32_t)seg.size() - 1;
    if (sys_ptr)
        for (size_t i = 0; i < seg.size(); ++i) sys_ptr[i] = seg[i];
    return RSC_OK;
}

rsc_status rsc_solve_batch_device(rsc_handle* h, int32_t nrhs, const double* d_B, double* d_X, double rtol,
                                  int32_t max_iter, int32_t* iters, double* final_relres, void* stream) {
    if (!h) return fail(nullptr, RSC_ERR_INVALID_ARG, "NULL handle");
    if (!d_B || !d_X || !iters || !final_relres || nrhs < 1)
        return fail(h, RSC_ERR_INVALID_ARG, "d_B, d_X, iters, final_relres and nrhs >= 1 are required");
    return guarded(h, [&]() -> rsc_status {
        if (!h->eng || !h->eng->factored()) return fail(h, RSC_ERR_STATE, "rsc_solve_batch_device before rsc_factor");
        std::vector<long long> seg;
        if (!system_ranges(h->sym, seg))
            return fail(h, RSC_ERR_INVALID_ARG, "independent systems do not occupy contiguous row ranges");
        std::vector<int> it(seg.size() - 1 > 0 ? (seg.size() - 1) * nrhs : 0);
        rsc_status st = h->eng->solve_batch_device(h->row_ptr, h->col_idx, h->val, seg, d_B, d_X, nrhs, rtol, max_iter,
                                                   it.data(), final_relres, stream);
        for (size_t q = 0; q < it.size(); ++q) iters[q] = it[q];
        if (st == RSC_ERR_NO_CONVERGENCE) return fail(h, st, "some systems did not reach rtol");
        return st;
    });
}

rsc_status rsc_pattern_outer_device(rsc_handle* h, const double* d_u, const double* d_v, double alpha,
                                    double* d_out, void* stream) {
    if (!h) return fail(nullptr, RSC_ERR_INVALID_ARG, "NULL handle");
    if (!d_u || !d_v || !d_out) return fail(h, RSC_ERR_INVALID_ARG, "d_u, d_v and d_out are required");
    return guarded(h, [&]() -> rsc_status {
        if (!h->eng) h->eng = new Engine(h->sym, h->opts);
        return h->eng->pattern_outer(h->row_ptr, h->col_idx, h->val, d_u, d_v, alpha, d_out, stream);
    });
}

rsc_status rsc_get_supernode_info(const rsc_handle* h, int32_t j, int32_t* info) {
    if (!h || !info) return fail(nullptr, RSC_ERR_INVALID_ARG, "NULL argument");
    if (j < 0 || j >= h->sym.M) return fail(const_cast<rsc_handle*>(h), RSC_ERR_INVALID_ARG, "j out of range");
    const auto& S = h->sym;
    info[0] = S.ncols(j);
    info[1] = S.nrows(j);
    info[2] = info[3] = info[4] = 0;
    info[5] = 1;
    info[6] = S.level[j];
    info[7] = S.kind[j];
    if (h->eng && h->eng->factored()) h->eng->node_info(j, info);
    return RSC_OK;
}

rsc_status rsc_get_supernode_blocks(const rsc_handle* h, int32_t j, double* LD, double* LO) {
    if (!h) return fail(nullptr, RSC_ERR_INVALID_ARG, "NULL handle");
    rsc_handle* hh = const_cast<rsc_handle*>(h);
    if (j < 0 || j >= h->sym.M) return fail(hh, RSC_ERR_INVALID_ARG, "j out of range");
    return guarded(hh, [&]() -> rsc_status {
        if (!h->eng || !h->eng->factored()) return fail(hh, RSC_ERR_STATE, "no factor");
        return h->eng->node_blocks(j, LD, LO);
    });
}

rsc_status rsc_get_stats(const rsc_handle* h, rsc_stats_t* out) {
    if (!h || !out) return fail(nullptr, RSC_ERR_INVALID_ARG, "NULL argument");
    std::memset(out, 0, sizeof(*out));
    out->n_supernodes = h->sym.M;
    out->n_levels = h->sym.nlevels;
    if (h->eng) h->eng->stats(out);
    return RSC_OK;
}

rsc_status rsc_profile(rsc_handle* h, int32_t enable, const char* kernels) {
    if (!h) return fail(nullptr, RSC_ERR_INVALID_ARG, "NULL handle");
    return guarded(h, [&]() -> rsc_status {
        if (!h->eng) h->eng = new Engine(h->sym, h->opts);
        h->eng->profile(enable, kernels);
        return RSC_OK;
    });
}

rsc_status rsc_get_kernel_profile(rsc_handle* h, char* json, int64_t len) {
    if (!h || !json || len <= 0) return fail(h, RSC_ERR_INVALID_ARG, "NULL argument");
    return guarded(h, [&]() -> rsc_status {
        std::string s = h->eng ? h->eng->profile_json() : std::string("{}");
        if ((int64_t)s.size() + 1 > len) return fail(h, RSC_ERR_INVALID_ARG, "buffer too small");
        std::memcpy(json, s.c_str(), s.size() + 1);
        return RSC_OK;
    });
}

rsc_status rsc_set_wait_limit(rsc_handle* h, int64_t polls) {
    if (!h) return fail(nullptr, RSC_ERR_INVALID_ARG, "NULL handle");
    if (polls < 0) return fail(h, RSC_ERR_INVALID_ARG, "polls must be >= 0");
    return guarded(h, [&]() -> rsc_status {
        if (!h->eng) h->eng = new Engine(h->sym, h->opts);
        h->eng->set_wait_limit(polls);
        return RSC_OK;
    });
}

rsc_status rsc_get_autotune(const rsc_handle* h, char* json, int64_t len) {
    rsc_handle* hh = const_cast<rsc_handle*>(h);
    if (!h || !json || len <= 0) return fail(hh, RSC_ERR_INVALID_ARG, "NULL argument");
    return guarded(hh, [&]() -> rsc_status {
        std::string s = h->eng ? h->eng->tuning_json() : std::string("{}");
        if ((int64_t)s.size() + 1 > len) return fail(hh, RSC_ERR_INVALID_ARG, "buffer too small");
        std::memcpy(json, s.c_str(), s.size() + 1);
        return RSC_OK;
    });
}

const char* rsc_last_error(const rsc_handle* h) {
    if (h) return h->err.c_str();
    return g_last_error.c_str();
}

void rsc_destroy(rsc_handle* h) {
    if (!h) return;
    try {
        delete h->eng;
    } catch (...) {
    }
    delete h;
}

}  // extern "C"
