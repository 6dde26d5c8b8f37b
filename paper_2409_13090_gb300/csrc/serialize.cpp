// Symbolic handle on disk (sc_symbolic_save / sc_symbolic_load in
// include/sc.h): analyze once, factor in later processes. The file holds the
// options, the plan settings and every host structure of the analysis; the
// device schedule is rebuilt on load from them (it is a function of them).
//
// Layout (little-endian, as on both supported hosts): 8-byte magic, uint32
// byte-order mark, uint32 version, the scalars, then each array as int64
// count, uint32 element size and the raw elements, then an FNV-1a 64-bit hash
// of everything before it.
#include <cstdio>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "sc_internal.h"

namespace {

constexpr char kMagic[8] = {'S', 'C', 'S', 'Y', 'M', 'B', 'O', 'L'};
constexpr uint32_t kByteOrder = 0x01020304u, kVersion = 1;

struct Writer {
    std::string buf;
    void raw(const void *p, size_t n) { buf.append(static_cast<const char *>(p), n); }
    template <typename T>
    void val(const T &v) {
        raw(&v, sizeof(T));
    }
    template <typename T>
    void vec(const std::vector<T> &v) {
        val<int64_t>((int64_t)v.size());
        val<uint32_t>((uint32_t)sizeof(T));
        raw(v.data(), v.size() * sizeof(T));
    }
};

struct Reader {
    const std::string &buf;
    size_t pos = 0;
    bool ok = true;
    explicit Reader(const std::string &b) : buf(b) {}
    bool raw(void *p, size_t n) {
        if (!ok || n > buf.size() - pos) return ok = false;
        std::memcpy(p, buf.data() + pos, n);
        pos += n;
        return true;
    }
    template <typename T>
    bool val(T &v) {
        return raw(&v, sizeof(T));
    }
    template <typename T>
    bool vec(std::vector<T> &v) {
        int64_t n = 0;
        uint32_t es = 0;
        if (!val(n) || !val(es) || es != sizeof(T) || n < 0 || (uint64_t)n > (buf.size() - pos) / sizeof(T))
            return ok = false;
        v.resize((size_t)n);
        return raw(v.data(), (size_t)n * sizeof(T));
    }
};

uint64_t fnv1a(const char *p, size_t n) {
    uint64_t h = 1469598103934665603ull;
    for (size_t i = 0; i < n; i++) {
        h ^= (unsigned char)p[i];
        h *= 1099511628211ull;
    }
    return h;
}

// the host structures in file order (one list for writing and reading)
template <typename F>
void arrays(sc_symbolic &s, F &&f) {
    f(s.colptr), f(s.rowind), f(s.perm), f(s.iperm), f(s.cparent), f(s.sup_ptr), f(s.sup_parent), f(s.level),
        f(s.gl_ptr), f(s.glbind), f(s.ri_ptr), f(s.relind), f(s.blk_ptr), f(s.blk_first), f(s.blk_size),
        f(s.blk_owner), f(s.rb_pair_ptr), f(s.rb_pair_P), f(s.rb_val_ptr), f(s.rb_val), f(s.lnz_off), f(s.lnz_ld),
        f(s.valmap), f(s.sup_of), f(s.csr_ptr), f(s.csr_col), f(s.csr_map);
}

// sizes that the device schedule and the kernels rely on
bool consistent(const sc_symbolic &s) {
    const int64_t n = s.n, ns = s.nsuper;
    if (n < 1 || ns < 1 || ns > n) return false;
    const sc_options &o = s.opt;
    if ((o.variant != SC_RLB && o.variant != SC_RL) || o.precision < SC_FP64 || o.precision > SC_TF32X3 ||
        o.chunk < 1 || o.chunk > 64 || o.spin_limit < 1 ||
        (o.deterministic != 0 && !(o.deterministic == 1 && o.variant == SC_RL)))
        return false;
    auto sz = [](const auto &v, int64_t want) { return (int64_t)v.size() == want; };
    if (!sz(s.colptr, n + 1) || !sz(s.perm, n) || !sz(s.iperm, n) || !sz(s.cparent, n) || !sz(s.sup_of, n) ||
        !sz(s.sup_ptr, ns + 1) || !sz(s.sup_parent, ns) || !sz(s.level, ns) || !sz(s.gl_ptr, ns + 1) ||
        !sz(s.ri_ptr, ns + 1) || !sz(s.blk_ptr, ns + 1) || !sz(s.rb_pair_ptr, ns + 1) || !sz(s.lnz_off, ns) ||
        !sz(s.lnz_ld, ns) || !sz(s.csr_ptr, n + 1))
        return false;
    if (s.colptr[0] != 0 || !sz(s.rowind, s.colptr[n]) || !sz(s.valmap, s.colptr[n])) return false;
    if (s.sup_ptr[0] != 0 || s.sup_ptr[ns] != n || s.gl_ptr[ns] != (int64_t)s.glbind.size() ||
        s.ri_ptr[ns] != (int64_t)s.relind.size() || s.blk_ptr[ns] != (int64_t)s.blk_first.size() ||
        !sz(s.blk_size, s.blk_ptr[ns]) || !sz(s.blk_owner, s.blk_ptr[ns]) ||
        s.rb_pair_ptr[ns] != (int64_t)s.rb_pair_P.size() || !sz(s.rb_val_ptr, (int64_t)s.rb_pair_P.size() + 1) ||
        s.rb_val_ptr.back() != (int64_t)s.rb_val.size() || s.csr_ptr[n] != (int64_t)s.csr_col.size() ||
        !sz(s.csr_map, s.csr_ptr[n]))
        return false;
    for (int64_t J = 0; J < ns; J++) {
        const int64_t m = s.gl_ptr[J + 1] - s.gl_ptr[J], w = s.sup_ptr[J + 1] - s.sup_ptr[J];
        if (w < 1 || m < w || s.lnz_ld[J] < w || s.lnz_off[J] < 0 || s.lnz_off[J] + m * s.lnz_ld[J] > s.lnz_size)
            return false;
    }
    for (int32_t g : s.glbind)
        if (g < 0 || g >= n) return false;
    for (int64_t p : s.valmap)
        if (p < 0 || p >= s.lnz_size) return false;
    for (int32_t c : s.csr_col)
        if (c < 0 || c >= n) return false;
    for (int64_t q : s.csr_map)
        if (q < 0 || q >= s.colptr[n]) return false;
    for (int32_t p : s.perm)
        if (p < 0 || p >= n) return false;
    return true;
}

}  // namespace

extern "C" int sc_symbolic_save(const sc_symbolic *s, const char *path) {
    if (!s) return -1;
    if (!path) return -2;
    if (s->poisoned) return SC_ERR_INTERNAL;
    try {
        Writer w;
        w.raw(kMagic, sizeof(kMagic));
        w.val(kByteOrder);
        w.val(kVersion);
        sc_options o = s->opt;
        o.user_perm = nullptr;
        o.tune = nullptr;
        o.threads = 0;  // how the analysis ran, not what it produced
        w.val(o);
        w.val(s->tune);
        w.val(s->n);
        w.val(s->nsuper);
        w.val(s->nnzL);
        w.val(s->lnz_size);
        w.val(s->flops);
        arrays(const_cast<sc_symbolic &>(*s), [&](auto &v) { w.vec(v); });
        const uint64_t h = fnv1a(w.buf.data(), w.buf.size());
        w.val(h);
        std::unique_ptr<FILE, int (*)(FILE *)> f(std::fopen(path, "wb"), &std::fclose);
        if (!f) return SC_ERR_IO;
        if (std::fwrite(w.buf.data(), 1, w.buf.size(), f.get()) != w.buf.size()) return SC_ERR_IO;
        if (std::fflush(f.get()) != 0) return SC_ERR_IO;
        return SC_OK;
    } catch (const std::bad_alloc &) {
        return SC_ERR_OOM;
    }
}

extern "C" int sc_symbolic_load(const char *path, sc_symbolic **out) {
    if (!path) return -1;
    if (!out) return -2;
    *out = nullptr;
    try {
        std::string buf;
        {
            std::unique_ptr<FILE, int (*)(FILE *)> f(std::fopen(path, "rb"), &std::fclose);
            if (!f) return SC_ERR_IO;
            char tmp[1 << 16];
            size_t got;
            while ((got = std::fread(tmp, 1, sizeof(tmp), f.get())) > 0) buf.append(tmp, got);
            if (std::ferror(f.get())) return SC_ERR_IO;
        }
        if (buf.size() < sizeof(kMagic) + 8 + sizeof(uint64_t)) return SC_ERR_IO;
        uint64_t h = 0;
        std::memcpy(&h, buf.data() + buf.size() - sizeof(h), sizeof(h));
        if (h != fnv1a(buf.data(), buf.size() - sizeof(h))) return SC_ERR_IO;
        buf.resize(buf.size() - sizeof(h));
        Reader r(buf);
        char magic[8];
        uint32_t order = 0, version = 0;
        if (!r.raw(magic, 8) || std::memcmp(magic, kMagic, 8) != 0 || !r.val(order) || order != kByteOrder ||
            !r.val(version) || version != kVersion)
            return SC_ERR_IO;
        auto s = std::make_unique<sc_symbolic>();
        r.val(s->opt);
        s->opt.user_perm = nullptr;
        s->opt.tune = nullptr;
        r.val(s->tune);
        r.val(s->n);
        r.val(s->nsuper);
        r.val(s->nnzL);
        r.val(s->lnz_size);
        r.val(s->flops);
        arrays(*s, [&](auto &v) { r.vec(v); });
        if (!r.ok || r.pos != buf.size()) return SC_ERR_IO;
        if (!sc::tune_valid(s->tune) || !consistent(*s)) return SC_ERR_IO;
        int rc = sc::build_schedule(s.get());
        if (rc) return rc;
        // every device address the schedule implies is checked before the
        // handle can reach a kernel
        if (sc_check_schedule(s.get(), nullptr, 0) != SC_OK) return SC_ERR_IO;
        *out = s.release();
        return SC_OK;
    } catch (const std::bad_alloc &) {
        return SC_ERR_OOM;
    }
}
