// builder.cpp -- the graph compiler (paper Sec. 2.2-2.3).
//
// Input: a registry of canonical labels.  Output: a bundle holding the
// generator stage records (a; i, j; alpha) and the commutator stage records
// (k; a, j; beta) of Eq. (graph-actions), grouped by output.
//
// Bounded memory (Sec. 2.3): the algebra is traversed twice.  The first
// traversal only counts records per output (and discovers the generator
// coordinates and the distinct exact factors); the arrays are then allocated
// at their final sizes and the second traversal writes every record straight
// into its slot.  Records of one output are finally sorted by (input 1,
// input 2), so the bundle is bitwise reproducible for any thread count.
#include <sys/resource.h>

#include "trace.h"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstring>
#include <map>
#include <mutex>
#include <set>
#include <stdexcept>
#include <string>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "algebra.h"
#include "bundle.h"
#include "cut.h"
#include "status.h"

namespace cut {

namespace {

struct LabelIndex {  // open addressing label -> registry index
    std::vector<uint64_t> keys;
    std::vector<int32_t> vals;
    uint64_t mask = 0;
    explicit LabelIndex(const std::vector<uint64_t> &labels) {
        size_t cap = 16;
        while (cap < 2 * labels.size()) cap <<= 1;
        keys.assign(cap, 0);
        vals.assign(cap, -1);
        mask = cap - 1;
        for (size_t i = 0; i < labels.size(); i++) {
            size_t p = hash(labels[i]) & mask;
            while (vals[p] >= 0) {
                if (keys[p] == labels[i]) throw std::invalid_argument("duplicate label in registry");
                p = (p + 1) & mask;
            }
            keys[p] = labels[i];
            vals[p] = (int32_t)i;
        }
    }
    static uint64_t hash(uint64_t k) {
        k ^= k >> 31; k *= 0x7fb5d329728ea185ULL;
        k ^= k >> 27; k *= 0x81dadef4bc2dd44dULL;
        return k ^ (k >> 33);
    }
    int32_t find(uint64_t k) const {
        size_t p = hash(k) & mask;
        while (vals[p] >= 0) {
            if (keys[p] == k) return vals[p];
            p = (p + 1) & mask;
        }
        return -1;
    }
};

// Stored factor of one commutator term (see cut.h conventions).
//  generator stage: eta += h_i h_j c G  ->  xi gets c (fermion) or c / i (Pauli)
//  commutator stage: [eta, X] += xi_a x_j c' O_k times 1 (fermion) or i (Pauli)
inline int gen_factor(int alg, const Term &t) {
    if (alg == 0) {
        if (t.re != 0) throw std::logic_error("Pauli generator term with a real part");
        return t.im;
    }
    if (t.im != 0) throw std::logic_error("fermion term with an imaginary part");
    return t.re;
}
inline int comm_factor(int alg, const Term &t) {
    if (alg == 0) {
        if (t.re != 0) throw std::logic_error("Pauli commutator term with a real part");
        return -t.im;
    }
    if (t.im != 0) throw std::logic_error("fermion term with an imaginary part");
    return t.re;
}

int hw_threads(int req) {
    if (req > 0) return req;
    unsigned h = std::thread::hardware_concurrency();
    return h ? (int)h : 4;
}

template <class F>
void parallel_chunks(int threads, int64_t total, int64_t chunk, F fn) {
    std::atomic<int64_t> next(0);
    std::vector<std::thread> pool;
    std::mutex emu;
    std::string err;
    for (int t = 0; t < threads; t++) {
        pool.emplace_back([&, t]() {
            try {
                for (;;) {
                    int64_t b = next.fetch_add(chunk);
                    if (b >= total) break;
                    fn(t, b, std::min(total, b + chunk));
                }
            } catch (const std::exception &e) {
                std::lock_guard<std::mutex> lk(emu);
                err = e.what();
                next.store(total);
            }
        });
    }
    for (auto &th : pool) th.join();
    if (!err.empty()) throw std::runtime_error(err);
}

struct Ctx {
    int alg = 0, nmodes = 0, max_rank = 0, threads = 1;
    std::vector<uint64_t> labels;
    std::vector<int32_t> diag_idx, off_idx;
    std::vector<std::vector<int32_t>> byC, byA;  // fermion: operands with p in C / in A
    std::unordered_map<uint32_t, std::vector<int32_t>> byCset, byAset;  // operands by exact C / A set
    int reg_rank = 0;                            // highest rank in the registry
    int diagnostics = 0;                         // keep outside-space records
    LabelIndex *reg = nullptr;
};

// Visit every generator-stage term: (g label, i, j, alpha) for diagonal i,
// off-diagonal j, with rank(g) <= max_rank.
template <class F>
void gen_terms(const Ctx &c, int64_t lo, int64_t hi, F emit) {
    Term buf[512];
    const int64_t no = (int64_t)c.off_idx.size();
    for (int64_t f = lo; f < hi; f++) {
        int32_t i = c.diag_idx[f / no], j = c.off_idx[f % no];
        int m = commutator(c.alg, c.labels[i], c.labels[j], buf);
        if (m < 0) throw std::invalid_argument("a product leaves the label range (boson degree > 31) or its factor is not an exact 32-bit integer");
        for (int t = 0; t < m; t++) {
            if (c.alg != 0 && rank_of(c.alg, buf[t].label) > c.max_rank) continue;
            emit(buf[t].label, i, j, gen_factor(c.alg, buf[t]));
        }
    }
}

// Visit every commutator-stage term for generator labels gl[lo..hi):
// (k registry index, a, j, beta) with O_k in the registry (projection P);
// with diagnostics, terms outside the registry go to emit_out(label, a, j,
// gamma) (the outside-space action of Eq. projected-flow).
struct NoOut {
    void operator()(uint64_t, int32_t, int32_t, int) const {}
};

template <class F, class FO = NoOut>
void comm_terms(const Ctx &c, const std::vector<uint64_t> &gl, int64_t lo, int64_t hi,
                std::vector<int32_t> &stamp, F emit, FO emit_out = FO()) {
    Term buf[512];
    const int32_t n = (int32_t)c.labels.size();
    for (int64_t a = lo; a < hi; a++) {
        uint64_t G = gl[a];
        auto visit = [&](int32_t j) {
            int m = commutator(c.alg, G, c.labels[j], buf);
            if (m < 0) throw std::invalid_argument("a product leaves the label range (boson degree > 31) or its factor is not an exact 32-bit integer");
            for (int t = 0; t < m; t++) {
                int32_t k = c.reg->find(buf[t].label);
                if (k >= 0) emit(k, (int32_t)a, j, comm_factor(c.alg, buf[t]));
                else if (c.diagnostics) emit_out(buf[t].label, (int32_t)a, j, comm_factor(c.alg, buf[t]));
            }
        };
        if (c.alg != 1) {
            for (int32_t j = 0; j < n; j++) visit(j);
        } else if (!c.diagnostics && popc(lo32(G)) >= c.reg_rank) {
            // A generator of the registry's top rank r: a term of G O_j has
            // rank r + r_j - |K| with K the contracted part of C_j, so it stays
            // within rank r only if every creator of O_j is contracted
            // (C_j subset of A_G); likewise A_j subset of C_G for O_j G.
            int32_t tag = (int32_t)a;
            uint32_t Ag = hi32(G), Cg = lo32(G);
            for (uint32_t S = Ag; S; S = (S - 1) & Ag) {
                auto it = c.byCset.find(S);
                if (it != c.byCset.end())
                    for (int32_t j : it->second)
                        if (stamp[j] != tag) { stamp[j] = tag; visit(j); }
            }
            for (uint32_t S = Cg; S; S = (S - 1) & Cg) {
                auto it = c.byAset.find(S);
                if (it != c.byAset.end())
                    for (int32_t j : it->second)
                        if (stamp[j] != tag) { stamp[j] = tag; visit(j); }
            }
        } else {
            // [G, O_j] vanishes unless an annihilator of G meets a creator of
            // O_j or a creator of G meets an annihilator of O_j.
            int32_t tag = (int32_t)a;
            uint32_t Ag = hi32(G), Cg = lo32(G);
            for (uint32_t s = Ag; s; s &= s - 1)
                for (int32_t j : c.byC[__builtin_ctz(s)])
                    if (stamp[j] != tag) { stamp[j] = tag; visit(j); }
            for (uint32_t s = Cg; s; s &= s - 1)
                for (int32_t j : c.byA[__builtin_ctz(s)])
                    if (stamp[j] != tag) { stamp[j] = tag; visit(j); }
        }
    }
}

// distinct exact factors seen by one thread
struct WeightSet {
    static constexpr int kR = 4096;
    std::vector<uint8_t> seen = std::vector<uint8_t>(2 * kR + 1, 0);
    std::set<int> other;
    void insert(int w) {
        if (w >= -kR && w <= kR) seen[w + kR] = 1;
        else other.insert(w);
    }
    void collect(std::set<int> &out) const {
        for (int v = -kR; v <= kR; v++)
            if (seen[v + kR]) out.insert(v);
        out.insert(other.begin(), other.end());
    }
};

inline bool gen_less(int alg, uint64_t x, uint64_t y) {
    int rx = rank_of(alg, x), ry = rank_of(alg, y);
    if (rx != ry) return rx < ry;
    return x < y;
}

void sort_segments(int threads, const std::vector<uint64_t> &rp, std::vector<uint32_t> &rec) {
    struct R { uint32_t w0, w1; };
    R *r = reinterpret_cast<R *>(rec.data());
    int64_t rows = (int64_t)rp.size() - 1;
    parallel_chunks(threads, rows, 64, [&](int, int64_t lo, int64_t hi) {
        for (int64_t k = lo; k < hi; k++)
            std::sort(r + rp[k], r + rp[k + 1], [](const R &x, const R &y) {
                uint32_t ax = x.w0 & kIndexMask, ay = y.w0 & kIndexMask;
                return ax != ay ? ax < ay : x.w1 < y.w1;
            });
    });
}

}  // namespace

// Build the whole graph in host memory.
void build_graph(const cut_build_opts &o, int64_t n, const uint64_t *labels, HostGraph &g,
                 cut_build_stats *st) {
    using clk = std::chrono::steady_clock;
    auto t0 = clk::now();
    TraceRange count("cut_build/count");
    Ctx c;
    c.alg = o.algebra;
    c.nmodes = o.nmodes;
    c.threads = hw_threads(o.threads);
    c.labels.assign(labels, labels + n);
    int reg_rank = 0;
    for (auto l : c.labels) {
        if (c.alg == 2) {
            if (o.nmodes > kPBModes) throw std::invalid_argument("Pauli-boson labels hold at most 6 modes");
            const uint64_t used_bits = (o.nmodes == kPBModes) ? ~0ull >> 2 : ((1ull << (2 + 10 * o.nmodes)) - 1);
            if (l & ~used_bits) throw std::invalid_argument("label uses a mode beyond nmodes");
        } else {
            uint32_t lo = lo32(l), hi = hi32(l);
            uint64_t modes = o.nmodes == 32 ? 0xFFFFFFFFull : ((1ull << o.nmodes) - 1);
            if ((lo & ~modes) || (hi & ~modes)) throw std::invalid_argument("label uses a mode beyond nmodes");
            if (c.alg == 1 && popc(lo) != popc(hi)) throw std::invalid_argument("fermion label is not number conserving");
            if (c.alg == 1 && popc(lo) == 0) throw std::invalid_argument("the identity is not a registry coordinate");
        }
        reg_rank = std::max(reg_rank, rank_of(c.alg, l));
    }
    c.diagnostics = o.diagnostics ? 1 : 0;
    // diagnostics need every generator term (eta exact); for fermions terms of
    // rank above the registry's cannot reach it otherwise.  Pauli-boson
    // generators are always kept exact (no rank lemma there: contractions
    // lower the boson degree).
    c.max_rank = o.max_rank > 0 ? o.max_rank : ((c.diagnostics || c.alg == 2) ? 64 : reg_rank);
    c.reg_rank = reg_rank;
    LabelIndex reg(c.labels);
    c.reg = &reg;
    for (int32_t i = 0; i < (int32_t)n; i++) (is_diagonal(c.alg, c.labels[i]) ? c.diag_idx : c.off_idx).push_back(i);
    if (c.alg == 1) {
        c.byC.assign(32, {});
        c.byA.assign(32, {});
        for (int32_t j = 0; j < (int32_t)n; j++) {
            for (uint32_t s = lo32(c.labels[j]); s; s &= s - 1) c.byC[__builtin_ctz(s)].push_back(j);
            for (uint32_t s = hi32(c.labels[j]); s; s &= s - 1) c.byA[__builtin_ctz(s)].push_back(j);
            c.byCset[lo32(c.labels[j])].push_back(j);
            c.byAset[hi32(c.labels[j])].push_back(j);
        }
    }
    const int T = c.threads;
    const int64_t gen_pairs = (int64_t)c.diag_idx.size() * (int64_t)c.off_idx.size();

    // ---- traversal 1a: generator coordinates and their factors
    std::vector<std::unordered_set<uint64_t>> tl_gen(T);
    std::vector<WeightSet> tl_w(T);
    parallel_chunks(T, gen_pairs, 4096, [&](int t, int64_t lo, int64_t hi) {
        gen_terms(c, lo, hi, [&](uint64_t gl, int32_t, int32_t, int w) {
            tl_gen[t].insert(gl);
            tl_w[t].insert(w);
        });
    });
    std::set<uint64_t> cand_set;
    for (auto &s : tl_gen) { cand_set.insert(s.begin(), s.end()); s.clear(); }
    std::vector<uint64_t> cand(cand_set.begin(), cand_set.end());
    cand_set.clear();
    std::sort(cand.begin(), cand.end(), [&](uint64_t x, uint64_t y) { return gen_less(c.alg, x, y); });

    // ---- traversal 1b: count commutator records per output; which
    //      generator coordinates reach the registry at all
    std::vector<uint32_t> comm_cnt(n, 0);
    std::vector<uint8_t> used(cand.size(), 0);
    std::vector<std::unordered_map<uint64_t, uint32_t>> tl_out(T);
    {
        std::vector<std::vector<int32_t>> stamps(T, std::vector<int32_t>(n, -1));
        parallel_chunks(T, (int64_t)cand.size(), 16, [&](int t, int64_t lo, int64_t hi) {
            comm_terms(
                c, cand, lo, hi, stamps[t],
                [&](int32_t k, int32_t a, int32_t, int w) {
                    __atomic_fetch_add(&comm_cnt[k], 1u, __ATOMIC_RELAXED);
                    __atomic_store_n(&used[a], (uint8_t)1, __ATOMIC_RELAXED);
                    tl_w[t].insert(w);
                },
                [&](uint64_t lab, int32_t a, int32_t, int w) {
                    tl_out[t][lab]++;
                    __atomic_store_n(&used[a], (uint8_t)1, __ATOMIC_RELAXED);
                    tl_w[t].insert(w);
                });
        });
    }
    // outside-space labels (diagnostics): sorted by rank, then label
    std::map<uint64_t, uint32_t> out_cnt_map;
    for (auto &m : tl_out) {
        for (auto &kv : m) out_cnt_map[kv.first] += kv.second;
        m.clear();
    }
    std::vector<uint64_t> out_labels;
    for (auto &kv : out_cnt_map) out_labels.push_back(kv.first);
    std::sort(out_labels.begin(), out_labels.end(), [&](uint64_t x, uint64_t y) { return gen_less(c.alg, x, y); });
    if ((int64_t)out_labels.size() > (int64_t)kIndexMask) throw std::invalid_argument("outside space beyond 2^24 labels");
    g.gen_labels.clear();
    for (size_t a = 0; a < cand.size(); a++)
        if (used[a]) g.gen_labels.push_back(cand[a]);
    cand.clear();
    cand.shrink_to_fit();
    LabelIndex gidx(g.gen_labels);
    const int64_t ng = (int64_t)g.gen_labels.size();

    // ---- traversal 1c: count generator records per (used) coordinate
    std::vector<uint32_t> gen_cnt(ng, 0);
    parallel_chunks(T, gen_pairs, 4096, [&](int, int64_t lo, int64_t hi) {
        gen_terms(c, lo, hi, [&](uint64_t gl, int32_t, int32_t, int) {
            int32_t a = gidx.find(gl);
            if (a >= 0) __atomic_fetch_add(&gen_cnt[a], 1u, __ATOMIC_RELAXED);
        });
    });

    // ---- exact factor table (integers here: den = 1), ascending
    std::set<int> wset;
    for (auto &s : tl_w) s.collect(wset);
    if (wset.size() > (size_t)kMaxCodes) throw std::runtime_error("more than 256 distinct factors");
    std::map<int, uint32_t> code;
    g.num.clear();
    g.den.clear();
    for (int w : wset) {
        code[w] = (uint32_t)g.num.size();
        g.num.push_back(w);
        g.den.push_back(1);
    }
    if (g.num.empty()) { g.num.push_back(0); g.den.push_back(1); }
    int32_t code_lut[2 * 4096 + 1];
    const int kLut = 4096;
    for (int v = -kLut; v <= kLut; v++) code_lut[v + kLut] = code.count(v) ? (int32_t)code[v] : -1;
    auto code_of = [&](int w) -> uint32_t {
        if (w >= -kLut && w <= kLut && code_lut[w + kLut] >= 0) return (uint32_t)code_lut[w + kLut];
        return code.at(w);
    };

    // ---- allocate final arrays
    g.algebra = c.alg;
    g.nmodes = c.nmodes;
    g.max_rank = c.max_rank;
    g.labels = c.labels;
    g.diag.resize(n);
    for (int64_t i = 0; i < n; i++) g.diag[i] = is_diagonal(c.alg, c.labels[i]) ? 1 : 0;
    g.rp[0].assign(ng + 1, 0);
    for (int64_t a = 0; a < ng; a++) g.rp[0][a + 1] = g.rp[0][a] + gen_cnt[a];
    g.rp[1].assign(n + 1, 0);
    for (int64_t k = 0; k < n; k++) g.rp[1][k + 1] = g.rp[1][k] + comm_cnt[k];
    if (ng > (int64_t)kIndexMask || n > (int64_t)kIndexMask) throw std::invalid_argument("index beyond 2^24");
    g.rec[0].assign(2 * g.rp[0][ng], 0);
    g.rec[1].assign(2 * g.rp[1][n], 0);
    g.out_labels = out_labels;
    const int64_t nout = (int64_t)out_labels.size();
    g.rp[2].assign(nout + 1, 0);
    for (int64_t q = 0; q < nout; q++) g.rp[2][q + 1] = g.rp[2][q] + out_cnt_map[out_labels[q]];
    g.rec[2].assign(2 * g.rp[2][nout], 0);
    out_cnt_map.clear();
    LabelIndex oidx(g.out_labels);
    auto t1 = clk::now();
    count.end();
    TraceRange write("cut_build/write");

    // ---- traversal 2: write every record into its final slot
    {
        std::vector<uint64_t> cur(g.rp[0].begin(), g.rp[0].end() - 1);
        uint32_t *rc = g.rec[0].data();
        parallel_chunks(T, gen_pairs, 4096, [&](int, int64_t lo, int64_t hi) {
            gen_terms(c, lo, hi, [&](uint64_t gl, int32_t i, int32_t j, int w) {
                int32_t a = gidx.find(gl);
                if (a < 0) return;
                uint64_t p = __atomic_fetch_add(&cur[a], 1ull, __ATOMIC_RELAXED);
                rc[2 * p] = (code_of(w) << kIndexBits) | (uint32_t)i;
                rc[2 * p + 1] = (uint32_t)j;
            });
        });
    }
    {
        std::vector<uint64_t> cur(g.rp[1].begin(), g.rp[1].end() - 1);
        std::vector<uint64_t> ocur(g.rp[2].begin(), g.rp[2].end() - 1);
        uint32_t *rc = g.rec[1].data();
        uint32_t *oc = g.rec[2].data();
        std::vector<std::vector<int32_t>> stamps(T, std::vector<int32_t>(n, -1));
        parallel_chunks(T, ng, 16, [&](int t, int64_t lo, int64_t hi) {
            comm_terms(
                c, g.gen_labels, lo, hi, stamps[t],
                [&](int32_t k, int32_t a, int32_t j, int w) {
                    uint64_t p = __atomic_fetch_add(&cur[k], 1ull, __ATOMIC_RELAXED);
                    rc[2 * p] = (code_of(w) << kIndexBits) | (uint32_t)a;
                    rc[2 * p + 1] = (uint32_t)j;
                },
                [&](uint64_t lab, int32_t a, int32_t j, int w) {
                    const int32_t q = oidx.find(lab);
                    uint64_t p = __atomic_fetch_add(&ocur[q], 1ull, __ATOMIC_RELAXED);
                    oc[2 * p] = (code_of(w) << kIndexBits) | (uint32_t)a;
                    oc[2 * p + 1] = (uint32_t)j;
                });
        });
    }
    sort_segments(T, g.rp[0], g.rec[0]);
    sort_segments(T, g.rp[1], g.rec[1]);
    sort_segments(T, g.rp[2], g.rec[2]);
    auto t2 = clk::now();
    write.end();
    if (st) {
        st->n = n;
        st->n_g = ng;
        st->R_g = g.R(0);
        st->R_L = g.R(1);
        st->n_codes = (int)g.num.size();
        st->seconds_count = std::chrono::duration<double>(t1 - t0).count();
        st->seconds_write = std::chrono::duration<double>(t2 - t1).count();
    }
}

}  // namespace cut

extern "C" cut_status cut_build(const cut_build_opts *opts, int64_t n, const uint64_t *labels,
                                const char *path, cut_build_stats *stats) {
    using namespace cut;
    if (!opts || !labels || !path || n <= 0) return set_error(CUT_ERR_INVALID_ARG, "cut_build: null argument or empty registry");
    if (opts->algebra != CUT_ALG_PAULI && opts->algebra != CUT_ALG_FERMION && opts->algebra != CUT_ALG_PAULI_BOSON)
        return set_error(CUT_ERR_INVALID_ARG, "cut_build: unknown algebra");
    if (opts->nmodes < 1 || opts->nmodes > 32) return set_error(CUT_ERR_INVALID_ARG, "cut_build: nmodes must be 1..32");
    auto t0 = std::chrono::steady_clock::now();
    TraceRange trace("cut_build");
    cut_build_stats local;
    memset(&local, 0, sizeof(local));
    try {
        HostGraph g;
        build_graph(*opts, n, labels, g, &local);
        int64_t bytes = 0;
        std::string e;
        {
            TraceRange tr("cut_build/store");
            e = write_bundle(g, path, &bytes);
        }
        if (!e.empty()) return set_error(CUT_ERR_IO, "cut_build: " + e);
        local.bytes_stored = bytes;
    } catch (const std::invalid_argument &e) {
        return set_error(CUT_ERR_INVALID_ARG, std::string("cut_build: ") + e.what());
    } catch (const std::bad_alloc &) {
        return set_error(CUT_ERR_OUT_OF_MEMORY, "cut_build: out of host memory");
    } catch (const std::exception &e) {
        return set_error(CUT_ERR_INVALID_ARG, std::string("cut_build: ") + e.what());
    }
    struct rusage ru;
    getrusage(RUSAGE_SELF, &ru);
    local.peak_rss_bytes = (int64_t)ru.ru_maxrss * 1024;
    local.seconds_total = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (stats) *stats = local;
    return set_ok();
}
