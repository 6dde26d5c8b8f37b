// Launch-plan autotuner (sc_tune in include/sc.h). The level schedule and the
// routing of Alg. 4/5's products follow from the structure; what is tuned are
// the depth of the trailing-update deferral inside supernodes (how many
// read-modify-write passes each target takes, and with which K), the
// thresholds that cut products into tiled tasks, device-loop items,
// tensor-core tiles or warp blocks, and the lookahead split. Each setting is
// timed by factoring the caller's matrix; coordinate descent over the fields
// of sc_tune_table, one pass, keeping a value only when it is clearly faster.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "numeric.h"
#include "sc_internal.h"

namespace {

struct Field {
    int32_t sc_tune_table::*member;
    std::vector<int32_t> values;
    bool schedule;  // changes the level schedule (rebuilt for the setting)
    bool tc_only;   // read only by the tensor-core routing
    bool rlb_only;  // read only by Alg. 5's loop split / the lookahead split
};

bool same_knobs(const sc_tune_table &a, const sc_tune_table &b) {
    const sc::Knobs x = sc::knobs_of(a), y = sc::knobs_of(b);
    return x.tile_min_entries == y.tile_min_entries && x.tile_min_k == y.tile_min_k &&
           x.loop_budget == y.loop_budget && x.lookahead == y.lookahead && x.tc_min_k == y.tc_min_k &&
           x.tc_wide_n == y.tc_wide_n && x.thin_dim == y.thin_dim && x.defer_width == y.defer_width && x.fused == y.fused &&
           x.tc_wide256 == y.tc_wide256 && x.solve_group == y.solve_group &&
           x.tc_multicast == y.tc_multicast;
}

double median(std::vector<double> v) {
    std::sort(v.begin(), v.end());
    const size_t n = v.size();
    return n % 2 ? v[n / 2] : 0.5 * (v[n / 2 - 1] + v[n / 2]);
}

// Factors with table t (schedule rebuilt first when `rebuild`): one untimed
// factorization (it also captures the graph), then `reps` timed ones.
int time_setting(sc_symbolic *s, const sc_tune_table &t, bool rebuild, const double *d_values, int precision,
                 int reps, cudaStream_t st, double *ms) {
    s->tune = t;
    int rc;
    if (rebuild && (rc = sc::build_schedule(s))) return rc;
    sc_numeric *h = nullptr;
    if ((rc = sc::numeric_create(s, precision, &h))) return rc;
    sc_factor_info info{};
    rc = sc::numeric_factor(h, d_values, 1, st, &info);
    std::vector<double> v;
    for (int r = 0; rc == 0 && r < reps; r++) {
        rc = sc::numeric_factor(h, d_values, 1, st, &info);
        v.push_back(info.factor_ms);
    }
    sc::numeric_free(h);
    if (rc) return rc;
    *ms = median(v);
    return SC_OK;
}

}  // namespace

extern "C" int sc_tune(sc_symbolic *s, const double *values, int values_on_device, int precision, int reps,
                       void *cuda_stream, sc_tune_table *best, int32_t *tried) {
    sc::NvtxRange range("sc_tune");
    if (!s) return -1;
    if (!values) return -2;
    if (values_on_device != 0 && values_on_device != 1) return -3;
    if (precision == -1) precision = s->opt.precision;
    if (precision < SC_FP64 || precision > SC_TF32X3) return -4;
    if (reps < 1 || reps > 15) return -5;
    if (!best) return -7;
    if (s->refs.load() > 0) return SC_ERR_IN_USE;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const bool tc = precision == SC_TF32 || precision == SC_TF32X3;
    const bool rlb = s->opt.variant == SC_RLB;

    // the values go to the device once; every setting factors from there
    const size_t nv = (size_t)s->colptr[s->n];
    double *owned = nullptr;
    const double *dv = values;
    if (!values_on_device) {
        if (cudaMalloc((void **)&owned, std::max<size_t>(nv, 1) * sizeof(double)) != cudaSuccess) return SC_ERR_OOM;
        if (cudaMemcpyAsync(owned, values, nv * sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            cudaFree(owned);
            return SC_ERR_CUDA;
        }
        dv = owned;
    }

    const sc_tune_table start = s->tune;
    sc_tune_table cur = start;
    int32_t count = 0;
    double best_ms = 0;
    int rc = time_setting(s, cur, false, dv, precision, reps, st, &best_ms);
    count++;
    const std::vector<Field> fields = {
        {&sc_tune_table::defer_width, {256, 512, 1024, 4096}, true, false, false},
        {&sc_tune_table::fused, {1, -1}, false, false, true},
        {&sc_tune_table::lookahead, {1, -1}, false, false, true},
        {&sc_tune_table::tile_min_entries, {512, 1024, 2048}, true, false, true},
        {&sc_tune_table::tile_min_k, {8, 16, 32}, true, false, true},
        {&sc_tune_table::loop_budget, {1 << 13, 1 << 15, 1 << 17}, true, false, true},
        {&sc_tune_table::thin_dim, {8, 4, -1}, false, false, false},
        {&sc_tune_table::tc_min_k, {32, 64, 128}, false, true, false},
        {&sc_tune_table::tc_wide_n, {64, 96, 128}, false, true, false},
        {&sc_tune_table::tc_wide256, {384, 1 << 20}, false, true, false},
        {&sc_tune_table::tc_multicast, {-1}, false, true, false},
    };
    bool dirty = false;  // the schedule in s is not the one of `cur`
    for (const Field &f : fields) {
        if (rc) break;
        if ((f.tc_only && !tc) || (f.rlb_only && !rlb)) continue;
        if (f.member == &sc_tune_table::lookahead && !s->opt.use_graph) continue;
        if (f.member == &sc_tune_table::fused && tc) continue;  // tensor-core precisions keep per-class launches
        for (int32_t v : f.values) {
            sc_tune_table cand = cur;
            cand.*f.member = v;
            if (same_knobs(cand, cur)) continue;
            double ms = 0;
            rc = time_setting(s, cand, f.schedule || dirty, dv, precision, reps, st, &ms);
            dirty = f.schedule;
            count++;
            if (rc) break;
            if (ms < 0.98 * best_ms) {
                best_ms = ms;
                cur = cand;
                dirty = false;
            }
        }
    }
    if (owned) cudaFree(owned);
    if (rc) {
        s->tune = start;
        sc::build_schedule(s);
        return rc;
    }
    s->tune = cur;
    if (dirty && (rc = sc::build_schedule(s))) return rc;
    *best = cur;
    best->factor_ms = best_ms;
    if (tried) *tried = count;
    return SC_OK;
}
