// C ABI of libsc (declared in include/sc.h): argument checks, handle
// ownership and error codes around the host analysis and the CUDA path.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>

#include "numeric.h"
#include "sc_internal.h"

extern "C" {

int sc_options_default(sc_options *o) {
    if (!o) return -1;
    std::memset(o, 0, sizeof(*o));
    o->ordering = SC_ORDER_NATURAL;
    o->nd_leaf = 8;
    o->user_perm = nullptr;
    o->pr = 1;
    o->variant = SC_RLB;
    o->precision = SC_FP64;
    o->chunk = 64;
    o->ir_tol = 1e-14;
    o->ir_maxit = 30;
    o->pivot_tau = 1.0 / 1024.0;
    o->spin_limit = 1 << 22;
    o->use_graph = 1;
    o->merge_frac = 0.0;
    return SC_OK;
}

int sc_analyze(int64_t n, const int64_t *colptr, const int32_t *rowind, const sc_options *o, sc_symbolic **out) {
    sc::NvtxRange range("sc_analyze");
    if (!out) return -5;
    *out = nullptr;
    sc_options def;
    sc_options_default(&def);
    const sc_options &opt = o ? *o : def;
    if (opt.variant != SC_RLB && opt.variant != SC_RL) return -4;
    if (opt.precision < SC_FP64 || opt.precision > SC_TF32X3) return -4;
    if (opt.chunk < 1 || opt.chunk > 64) return -4;
    if (!(opt.merge_frac >= 0.0)) return -4;
    if (opt.tune && !sc::tune_valid(*opt.tune)) return -4;
    if (opt.deterministic != 0 && !(opt.deterministic == 1 && opt.variant == SC_RL)) return -4;
    if (opt.threads < 0 || opt.threads > 1024) return -4;
    try {
        return sc::analyze_impl(n, colptr, rowind, opt, out);
    } catch (const std::bad_alloc &) {
        return SC_ERR_OOM;
    }
}

int sc_symbolic_export(const sc_symbolic *s, sc_symbolic_view *v) {
    if (!s) return -1;
    if (!v) return -2;
    v->n = s->n;
    v->nsuper = s->nsuper;
    v->nnzL = s->nnzL;
    v->nblocks = (int64_t)s->blk_first.size();
    v->npairs = (int64_t)s->rb_pair_P.size();
    v->flops = s->flops;
    v->perm = s->perm.data();
    v->sup_ptr = s->sup_ptr.data();
    v->sup_parent = s->sup_parent.data();
    v->gl_ptr = s->gl_ptr.data();
    v->glbind = s->glbind.data();
    v->ri_ptr = s->ri_ptr.data();
    v->relind = s->relind.data();
    v->blk_ptr = s->blk_ptr.data();
    v->blk_first = s->blk_first.data();
    v->blk_size = s->blk_size.data();
    v->blk_owner = s->blk_owner.data();
    v->rb_pair_ptr = s->rb_pair_ptr.data();
    v->rb_pair_P = s->rb_pair_P.data();
    v->rb_val_ptr = s->rb_val_ptr.data();
    v->rb_val = s->rb_val.data();
    v->level = s->level.data();
    v->cparent = s->cparent.data();
    return SC_OK;
}

int sc_relind_compose(const int32_t *rJC, int64_t lenJC, const int32_t *rCP, int64_t lenCP, int32_t *out) {
    return sc::compose_relind(rJC, lenJC, rCP, lenCP, out);
}

int sc_symbolic_free(sc_symbolic *s) {
    if (!s) return SC_OK;
    if (s->refs.load() > 0) return SC_ERR_IN_USE;
    delete s;
    return SC_OK;
}

int sc_factor(sc_symbolic *s, const double *values, int values_on_device, int precision, void *cuda_stream,
              sc_numeric **out, sc_factor_info *info) {
    sc::NvtxRange range("sc_factor");
    if (!s) return -1;
    if (!values) return -2;
    if (values_on_device != 0 && values_on_device != 1) return -3;
    if (precision == -1) precision = s->opt.precision;
    if (precision < SC_FP64 || precision > SC_TF32X3) return -4;
    if (!out) return -6;
    *out = nullptr;
    sc_numeric *h = nullptr;
    int rc;
    try {
        rc = sc::numeric_create(s, precision, &h);
    } catch (const std::bad_alloc &) {
        return SC_ERR_OOM;
    }
    if (rc) return rc;
    rc = sc::numeric_factor(h, values, values_on_device, (cudaStream_t)cuda_stream, info);
    if (rc < 0) {
        sc::numeric_free(h);
        return rc;
    }
    *out = h;
    return rc;
}

int sc_factor_batch(int count, sc_symbolic *const *syms, const double *const *values, int values_on_device,
                    int precision, void *cuda_stream, sc_symbolic **batch_sym, sc_numeric **out,
                    sc_factor_info *info) {
    sc::NvtxRange range("sc_factor_batch");
    if (count < 1) return -1;
    if (!syms) return -2;
    if (!values) return -3;
    if (values_on_device != 0 && values_on_device != 1) return -4;
    if (precision < SC_FP64 || precision > SC_TF32X3) return -5;
    if (!batch_sym) return -7;
    if (!out) return -8;
    *batch_sym = nullptr;
    *out = nullptr;
    for (int i = 0; i < count; i++)
        if (!syms[i] || !values[i]) return -2;
    sc_symbolic *b = nullptr;
    int rc = sc_analyze_batch(count, syms, &b);
    if (rc) return rc;
    // the batch's values: the matrices' values concatenated in order
    int64_t total = 0;
    for (int i = 0; i < count; i++) total += (int64_t)syms[i]->valmap.size();
    cudaStream_t st = (cudaStream_t)cuda_stream;
    double *d_vals = nullptr;
    if (cudaMalloc((void **)&d_vals, (size_t)std::max<int64_t>(1, total) * sizeof(double)) != cudaSuccess) {
        sc_symbolic_free(b);
        return SC_ERR_OOM;
    }
    int64_t off = 0;
    for (int i = 0; i < count && rc == SC_OK; i++) {
        const int64_t nnz = (int64_t)syms[i]->valmap.size();
        if (cudaMemcpyAsync(d_vals + off, values[i], nnz * sizeof(double),
                            values_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st) != cudaSuccess)
            rc = SC_ERR_CUDA;
        off += nnz;
    }
    if (rc == SC_OK) rc = sc_factor(b, d_vals, 1, precision, cuda_stream, out, info);
    cudaStreamSynchronize(st);
    cudaFree(d_vals);
    if (rc < 0) {
        sc_symbolic_free(b);
        return rc;
    }
    *batch_sym = b;
    return rc;
}

int sc_refactor(sc_numeric *h, const double *values, int values_on_device, void *cuda_stream, sc_factor_info *info) {
    sc::NvtxRange range("sc_refactor");
    if (!h) return -1;
    if (!values) return -2;
    if (values_on_device != 0 && values_on_device != 1) return -3;
    return sc::numeric_factor(h, values, values_on_device, (cudaStream_t)cuda_stream, info);
}

int sc_solve(sc_numeric *h, int64_t nrhs, const double *B, int64_t ldb, double *X, int64_t ldx, int on_device,
             void *cuda_stream, sc_solve_info *info) {
    sc::NvtxRange range("sc_solve");
    if (!h) return -1;
    if (nrhs < 1) return -2;
    if (!B) return -3;
    if (ldb < h->sym->n) return -4;
    if (!X || X == B) return -5;
    if (ldx < h->sym->n) return -6;
    if (on_device != 0 && on_device != 1) return -7;
    try {
        return sc::numeric_solve(h, nrhs, B, ldb, X, ldx, on_device, (cudaStream_t)cuda_stream, info);
    } catch (const std::bad_alloc &) {
        return SC_ERR_OOM;
    }
}

int sc_numeric_export_L(const sc_numeric *h, double *out) {
    if (!h) return -1;
    if (!out) return -2;
    return sc::numeric_export_L(h, out);
}

int sc_numeric_view(const sc_numeric *h, sc_factor_view *v) {
    if (!h) return -1;
    if (!v) return -2;
    if (h->last_stream && cudaStreamSynchronize(h->last_stream) != cudaSuccess) return SC_ERR_CUDA;
    const sc_symbolic *s = h->sym;
    v->lnz = h->d_lnz;
    v->elt = (int32_t)h->elt;
    v->precision = h->precision;
    v->size = s->lnz_size;
    v->nsuper = s->nsuper;
    v->panel_off = s->lnz_off.data();
    v->panel_ld = s->lnz_ld.data();
    return SC_OK;
}

int sc_factor_profile(sc_numeric *h, const double *values, int values_on_device, void *cuda_stream, double *ms,
                      double *flops, int32_t *launches) {
    if (!h) return -1;
    if (!values) return -2;
    if (values_on_device != 0 && values_on_device != 1) return -3;
    if (!ms) return -5;
    if (!flops) return -6;
    if (!launches) return -7;
    return sc::numeric_profile(h, values, values_on_device, (cudaStream_t)cuda_stream, ms, flops, launches);
}

int sc_plan_stats(const sc_symbolic *s, int precision, int64_t *out, int nout) {
    if (!s) return -1;
    if (precision < SC_FP64 || precision > SC_TF32X3) return -2;
    if (!out) return -3;
    return sc::plan_stats(s, precision, out, nout);
}

int sc_test_stall_solve(sc_numeric *h, int64_t chunk) {
    if (!h) return -1;
    if (chunk < 0 || chunk > INT32_MAX) return -2;
    h->stall_chunk = (int32_t)chunk;
    return SC_OK;
}

int sc_test_stall_factor(sc_numeric *h, int64_t chunk) {
    if (!h) return -1;
    if (chunk < 0 || chunk > INT32_MAX) return -2;
    h->stall_factor_chunk = (int32_t)chunk;
    return SC_OK;
}

void sc_numeric_free(sc_numeric *h) { sc::numeric_free(h); }

const char *sc_strerror(int code) {
    if (code == SC_OK) return "success";
    if (code > 0) return "matrix is not positive definite (pivot of the reported column is not positive)";
    switch (code) {
        case SC_ERR_CUDA: return "a CUDA runtime call failed";
        case SC_ERR_TIMEOUT: return "a bounded device-side wait gave up";
        case SC_ERR_NOT_CONVERGED: return "iterative refinement did not reach the tolerance";
        case SC_ERR_OOM: return "out of memory";
        case SC_ERR_IN_USE: return "symbolic handle still referenced by numeric handles";
        case SC_ERR_INTERNAL: return "internal consistency check failed";
        case SC_ERR_UNSUPPORTED: return "option not supported by this library";
        case SC_ERR_IO: return "file not written or read, or not a valid symbolic file";
        default: break;
    }
    if (code < 0 && code > -100) return "invalid argument (argument index = -code)";
    return "unknown error";
}

const char *sc_build_info(void) { return "libsc sm_103a"; }

}  // extern "C"
