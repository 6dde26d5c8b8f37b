// Batched analysis: many independent matrices factored as one block-diagonal
// problem. The supernodal forest of the batch is the union of the matrices'
// trees, so the chunk levels (heights) line up across matrices and every level
// of every matrix runs in the same launch of the level sequence.
#include <algorithm>

#include "sc_internal.h"

namespace {

template <typename T>
void append_shift(std::vector<T> &dst, const std::vector<T> &src, T shift, bool keep_negative = false) {
    for (T v : src) dst.push_back((keep_negative && v < 0) ? v : (T)(v + shift));
}

}  // namespace

extern "C" int sc_analyze_batch(int count, sc_symbolic *const *syms, sc_symbolic **out) {
    sc::NvtxRange range("sc_analyze_batch");
    if (count < 1) return -1;
    if (!syms) return -2;
    if (!out) return -3;
    *out = nullptr;
    for (int i = 0; i < count; i++)
        if (!syms[i]) return -2;
    try {
        auto b = new sc_symbolic();
        b->opt = syms[0]->opt;
        b->tune = syms[0]->tune;
        int64_t n0 = 0, ns0 = 0, nnz0 = 0, gl0 = 0, ri0 = 0, blk0 = 0, pair0 = 0, val0 = 0;
        b->colptr.push_back(0);
        b->sup_ptr.push_back(0);
        b->gl_ptr.push_back(0);
        b->ri_ptr.push_back(0);
        b->blk_ptr.push_back(0);
        b->rb_pair_ptr.push_back(0);
        b->rb_val_ptr.push_back(0);
        for (int i = 0; i < count; i++) {
            const sc_symbolic *s = syms[i];
            if (s->opt.variant != b->opt.variant || s->opt.deterministic != b->opt.deterministic) {
                delete b;
                return -2;
            }
            int64_t n = s->n;
            for (int64_t j = 1; j <= n; j++) b->colptr.push_back(s->colptr[j] + nnz0);
            append_shift<int32_t>(b->rowind, s->rowind, (int32_t)n0);
            append_shift<int32_t>(b->perm, s->perm, (int32_t)n0);
            append_shift<int32_t>(b->iperm, s->iperm, (int32_t)n0);
            append_shift<int32_t>(b->cparent, s->cparent, (int32_t)n0, true);
            for (int64_t J = 1; J <= s->nsuper; J++) b->sup_ptr.push_back(s->sup_ptr[J] + (int32_t)n0);
            append_shift<int32_t>(b->sup_parent, s->sup_parent, (int32_t)ns0, true);
            b->level.insert(b->level.end(), s->level.begin(), s->level.end());
            for (int64_t J = 1; J <= s->nsuper; J++) b->gl_ptr.push_back(s->gl_ptr[J] + gl0);
            append_shift<int32_t>(b->glbind, s->glbind, (int32_t)n0);
            for (int64_t J = 1; J <= s->nsuper; J++) b->ri_ptr.push_back(s->ri_ptr[J] + ri0);
            b->relind.insert(b->relind.end(), s->relind.begin(), s->relind.end());
            for (int64_t J = 1; J <= s->nsuper; J++) b->blk_ptr.push_back(s->blk_ptr[J] + blk0);
            append_shift<int32_t>(b->blk_first, s->blk_first, (int32_t)n0);
            b->blk_size.insert(b->blk_size.end(), s->blk_size.begin(), s->blk_size.end());
            append_shift<int32_t>(b->blk_owner, s->blk_owner, (int32_t)ns0);
            for (int64_t J = 1; J <= s->nsuper; J++) b->rb_pair_ptr.push_back(s->rb_pair_ptr[J] + pair0);
            append_shift<int32_t>(b->rb_pair_P, s->rb_pair_P, (int32_t)ns0);
            for (size_t q = 1; q < s->rb_val_ptr.size(); q++) b->rb_val_ptr.push_back(s->rb_val_ptr[q] + val0);
            b->rb_val.insert(b->rb_val.end(), s->rb_val.begin(), s->rb_val.end());
            append_shift<int32_t>(b->sup_of, s->sup_of, (int32_t)ns0);
            append_shift<int32_t>(b->csr_col, s->csr_col, (int32_t)n0);
            append_shift<int64_t>(b->csr_map, s->csr_map, nnz0);
            b->nnzL += s->nnzL;
            b->flops += s->flops;
            n0 += n;
            ns0 += s->nsuper;
            nnz0 += (int64_t)s->rowind.size();
            gl0 += (int64_t)s->glbind.size();
            ri0 += (int64_t)s->relind.size();
            blk0 += (int64_t)s->blk_first.size();
            pair0 += (int64_t)s->rb_pair_P.size();
            val0 += (int64_t)s->rb_val.size();
        }
        // row pointers of the block-diagonal CSR
        b->csr_ptr.assign(1, 0);
        for (int i = 0; i < count; i++) {
            const sc_symbolic *s = syms[i];
            int64_t base = b->csr_ptr.back();
            for (int64_t r = 1; r <= s->n; r++) b->csr_ptr.push_back(base + s->csr_ptr[r]);
        }
        b->n = n0;
        b->nsuper = ns0;
        // factor storage layout and value map of the combined problem
        b->lnz_off.resize(ns0);
        b->lnz_ld.resize(ns0);
        int64_t off = 0, J0 = 0, p0 = 0;
        for (int i = 0; i < count; i++) {
            const sc_symbolic *s = syms[i];
            off = (off + 31) / 32 * 32;
            for (int64_t J = 0; J < s->nsuper; J++) {
                b->lnz_off[J0 + J] = off + s->lnz_off[J];
                b->lnz_ld[J0 + J] = s->lnz_ld[J];
            }
            for (int64_t p = 0; p < (int64_t)s->valmap.size(); p++) b->valmap.push_back(off + s->valmap[p]);
            off += s->lnz_size;
            J0 += s->nsuper;
            p0 += (int64_t)s->valmap.size();
        }
        b->lnz_size = (off + 31) / 32 * 32;
        int rc = sc::build_schedule(b);
        if (rc) {
            delete b;
            return rc;
        }
        *out = b;
        return SC_OK;
    } catch (const std::bad_alloc &) {
        return SC_ERR_OOM;
    }
}
