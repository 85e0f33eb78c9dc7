// sssp_tune.cu -- autotuner of the round kernels' launch shape (hub degree,
// chunk size, CTAs per SM, cluster-tail limit) and the tuning cache keyed
// by graph class.  None of these parameters changes a result: they only
// decide how a round's work is spread over warps, CTAs and the cluster
// kernel, so the tuner is free to time any of them.  The paper has no
// counterpart.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>

#include "sssp_engine.h"

using namespace sssp;
using namespace sssp::engine;

namespace {

// ------------------------------------------------------------ the cache

struct TuneCache {
    std::mutex mu;
    bool opened = false;
    std::string path;                        // empty: in memory only
    std::map<std::string, sssp_tuning> map;
};
TuneCache& cache() {
    static TuneCache c;
    return c;
}

bool valid_tuning(const sssp_tuning& t) {
    return t.hub_degree >= 1 && t.hub_degree <= (1u << 20) && t.chunk_edges >= 32 &&
           t.chunk_edges <= (1u << 20) && t.chunk_edges % 32 == 0 && t.ctas_per_sm <= 64;
}

// A minimal reader for the file this module writes: an object of objects of
// unsigned integers.  Returns false on malformed input.
struct Reader {
    const char* p;
    const char* e;
    void ws() {
        while (p < e && (*p == ' ' || *p == '\n' || *p == '\r' || *p == '\t')) ++p;
    }
    bool lit(char c) {
        ws();
        if (p < e && *p == c) {
            ++p;
            return true;
        }
        return false;
    }
    bool str(std::string& out) {
        ws();
        if (p >= e || *p != '"') return false;
        const char* q = ++p;
        while (p < e && *p != '"') {
            if (*p == '\\') return false;
            ++p;
        }
        if (p >= e) return false;
        out.assign(q, p - q);
        ++p;
        return true;
    }
    bool num(unsigned long long& v) {
        ws();
        if (p >= e || *p < '0' || *p > '9') return false;
        v = 0;
        while (p < e && *p >= '0' && *p <= '9') {
            v = v * 10 + (unsigned long long)(*p - '0');
            if (v > 0xFFFFFFFFull) return false;
            ++p;
        }
        return true;
    }
};

bool parse(const std::string& text, std::map<std::string, sssp_tuning>& out) {
    Reader r{text.data(), text.data() + text.size()};
    if (!r.lit('{')) return false;
    if (r.lit('}')) return true;
    do {
        std::string key;
        if (!r.str(key) || !r.lit(':') || !r.lit('{')) return false;
        sssp_tuning t{};
        if (!r.lit('}')) {
            do {
                std::string f;
                unsigned long long v = 0;
                if (!r.str(f) || !r.lit(':') || !r.num(v)) return false;
                if (f == "hub_degree") t.hub_degree = (u32)v;
                else if (f == "chunk_edges") t.chunk_edges = (u32)v;
                else if (f == "ctas_per_sm") t.ctas_per_sm = (u32)v;
                else if (f == "tail_items") t.tail_items = (u32)v;
            } while (r.lit(','));
            if (!r.lit('}')) return false;
        }
        if (!valid_tuning(t)) return false;
        out[key] = t;
    } while (r.lit(','));
    if (!r.lit('}')) return false;
    r.ws();
    return r.p == r.e;
}

// Loads `path` into the cache (caller holds the lock).
int load_locked(TuneCache& c, const char* path) {
    c.map.clear();
    c.path = path ? path : "";
    c.opened = true;
    if (!path) return SSSP_OK;
    FILE* f = fopen(path, "rb");
    if (!f) return SSSP_OK;                  // no file yet: an empty cache
    std::string text;
    char buf[4096];
    size_t k;
    while ((k = fread(buf, 1, sizeof(buf), f)) > 0) text.append(buf, k);
    fclose(f);
    std::map<std::string, sssp_tuning> m;
    if (!parse(text, m)) return SSSP_E_INVAL;
    c.map.swap(m);
    return SSSP_OK;
}

void open_default_locked(TuneCache& c) {
    if (c.opened) return;
    const char* env = getenv("SSSP_TUNE_CACHE");
    if (load_locked(c, env && *env ? env : nullptr) != SSSP_OK) c.map.clear();
}

// Writes the cache back to its file (caller holds the lock): a temporary
// file renamed over the old one.
int store_locked(const TuneCache& c) {
    if (c.path.empty()) return SSSP_OK;
    const std::string tmp = c.path + ".tmp";
    FILE* f = fopen(tmp.c_str(), "wb");
    if (!f) return SSSP_E_INVAL;
    fputs("{", f);
    bool first = true;
    for (const auto& kv : c.map) {
        const sssp_tuning& t = kv.second;
        fprintf(f,
                "%s\n \"%s\": {\"hub_degree\": %u, \"chunk_edges\": %u, \"ctas_per_sm\": %u, "
                "\"tail_items\": %u}",
                first ? "" : ",", kv.first.c_str(), t.hub_degree, t.chunk_edges, t.ctas_per_sm,
                t.tail_items);
        first = false;
    }
    fputs("\n}\n", f);
    const bool ok = fclose(f) == 0;
    if (!ok || rename(tmp.c_str(), c.path.c_str()) != 0) return SSSP_E_INVAL;
    return SSSP_OK;
}

u32 log2_ceil(u64 x) {
    u32 b = 0;
    while (b < 64 && (1ull << b) < x) ++b;
    return b;
}

// ---------------------------------------------------------- the sweeps

constexpr u32 kHubs[] = {128, 256, 512, 1024};
constexpr u32 kChunks[] = {512, 1024, 2048};
constexpr u32 kTailItems[] = {0, 128, 256, 512, 1024, 2048};
constexpr u32 kCtas[] = {0, 1, 2, 4};

bool same(const sssp_tuning& a, const sssp_tuning& b) {
    return a.hub_degree == b.hub_degree && a.chunk_edges == b.chunk_edges &&
           a.ctas_per_sm == b.ctas_per_sm && a.tail_items == b.tail_items;
}

// Coordinate descent from `start`: each parameter group in turn, keeping a
// candidate when it is at least 0.5% faster.  time(t, &ms) measures one
// candidate.
template <class F>
int sweep(const sssp_tuning& start, F time, sssp_tune_result* out) {
    sssp_tuning best = start;
    double best_ms = 0;
    RC(time(best, &best_ms));
    const double start_ms = best_ms;
    u32 evaluated = 1;
    auto consider = [&](const sssp_tuning& t) -> int {
        if (same(t, best)) return SSSP_OK;
        double ms = 0;
        RC(time(t, &ms));
        ++evaluated;
        if (ms < best_ms * 0.995) {
            best = t;
            best_ms = ms;
        }
        return SSSP_OK;
    };
    const sssp_tuning g0 = best;
    for (u32 hub : kHubs)
        for (u32 ch : kChunks) {
            sssp_tuning t = g0;
            t.hub_degree = hub;
            t.chunk_edges = ch;
            RC(consider(t));
        }
    const sssp_tuning g1 = best;
    for (u32 ti : kTailItems) {
        sssp_tuning t = g1;
        t.tail_items = ti;
        RC(consider(t));
    }
    const sssp_tuning g2 = best;
    for (u32 cp : kCtas) {
        sssp_tuning t = g2;
        t.ctas_per_sm = cp;
        RC(consider(t));
    }
    if (out) {
        out->best = best;
        out->start_ms = start_ms;
        out->best_ms = best_ms;
        out->evaluated = evaluated;
        out->reserved = 0;
    }
    return SSSP_OK;
}

sssp_tuning tuning_of(const sssp_graph* h) {
    sssp_tuning t{};
    t.hub_degree = h->opt.hub_degree;
    t.chunk_edges = h->opt.chunk_edges;
    t.ctas_per_sm = h->opt.ctas_per_sm;
    t.tail_items = h->tail_items;
    return t;
}

// Sets a tuning on a handle (caller holds h->mu and the device).
int set_locked(sssp_graph* h, const sssp_tuning& t) {
    h->opt.hub_degree = t.hub_degree;
    h->opt.chunk_edges = t.chunk_edges;
    h->opt.ctas_per_sm = t.ctas_per_sm;
    h->tail_items = t.tail_items;
    return apply_tuning(h);
}

}  // namespace

namespace sssp {
namespace engine {

void graph_key(const sssp_graph* h, char* buf, size_t cap) {
    sssp_tune_key(h->n, h->m, h->max_out, h->max_in, h->wmax, buf, cap);
}

void batch_key(const sssp_handle* g, u32 k, char* buf, size_t cap) {
    u64 sn = 0, sm = 0;
    u32 mx = 0;
    bool narrow = true;
    for (u32 i = 0; i < k; ++i) {
        sn += g[i]->n;
        sm += g[i]->m;
        mx = std::max(mx, g[i]->n);
        narrow = narrow && g[i]->narrow;
    }
    snprintf(buf, cap, "batch.k%u.n%u.m%u.x%u.%c", log2_ceil(k), log2_ceil(sn), log2_ceil(sm),
             log2_ceil(mx), narrow ? 'c' : 'w');
}

int tune_cache_find(const char* key, sssp_tuning* out) { return sssp_tune_cache_get(key, out); }

// The tuning a new graph starts with: the cache's entry for its class when
// the options left the choice to the library, then the cluster-tail limits
// from the environment (SSSP_TAIL_ITEMS), which overrides.
void resolve_tuning(sssp_graph* h) {
    if (h->tune_auto) {
        char key[96];
        graph_key(h, key, sizeof(key));
        sssp_tuning t{};
        if (tune_cache_find(key, &t) == SSSP_OK) {
            h->opt.hub_degree = t.hub_degree;
            h->opt.chunk_edges = t.chunk_edges;
            h->opt.ctas_per_sm = t.ctas_per_sm;
            h->tail_items = t.tail_items;
        }
    }
    if (const char* v = getenv("SSSP_TAIL_ITEMS")) h->tail_items = (u32)strtoul(v, nullptr, 10);
}

}  // namespace engine
}  // namespace sssp

extern "C" {

int sssp_tune_key(uint32_t n, uint64_t m, uint32_t max_out_degree, uint32_t max_in_degree,
                  uint32_t max_weight, char* key, size_t cap) {
    if (!key || cap < 96) return SSSP_E_INVAL;
    // Average degree in half powers of two: round(2 log2(m / n)).
    const double avg = n ? (double)m / (double)n : 0.0;
    const int d2 = avg > 0 ? (int)std::lround(2.0 * std::log2(avg)) : -99;
    const bool narrow = (unsigned __int128)n * max_weight < kNarrowLimit;
    snprintf(key, cap, "graph.n%u.d%d.o%u.i%u.w%u.%c", log2_ceil(n), d2, log2_ceil(max_out_degree),
             log2_ceil(max_in_degree), log2_ceil(max_weight), narrow ? 'c' : 'w');
    return SSSP_OK;
}

int sssp_graph_key(sssp_handle h, char* key, size_t cap) {
    if (!h || !key || cap < 96) return SSSP_E_INVAL;
    graph_key(h, key, cap);
    return SSSP_OK;
}

int sssp_batch_key(const sssp_handle* g, uint32_t k, char* key, size_t cap) {
    if (!g || k == 0 || !key || cap < 96) return SSSP_E_INVAL;
    for (u32 i = 0; i < k; ++i)
        if (!g[i]) return SSSP_E_INVAL;
    batch_key(g, k, key, cap);
    return SSSP_OK;
}

int sssp_tune_cache_open(const char* path) {
    TuneCache& c = cache();
    std::lock_guard<std::mutex> lk(c.mu);
    const int rc = load_locked(c, path);
    if (rc != SSSP_OK) {
        c.map.clear();
        c.path.clear();
    }
    return rc;
}

int sssp_tune_cache_get(const char* key, sssp_tuning* out) {
    if (!key || !out) return SSSP_E_INVAL;
    TuneCache& c = cache();
    std::lock_guard<std::mutex> lk(c.mu);
    open_default_locked(c);
    auto it = c.map.find(key);
    if (it == c.map.end()) return SSSP_E_NOT_FOUND;
    *out = it->second;
    return SSSP_OK;
}

int sssp_tune_cache_put(const char* key, const sssp_tuning* t) {
    if (!key || !*key || !t || !valid_tuning(*t) || strchr(key, '"') || strchr(key, '\\'))
        return SSSP_E_INVAL;
    TuneCache& c = cache();
    std::lock_guard<std::mutex> lk(c.mu);
    open_default_locked(c);
    c.map[key] = *t;
    return store_locked(c);
}

int sssp_get_tuning(sssp_handle h, sssp_tuning* out) {
    if (!h || !out) return SSSP_E_INVAL;
    std::lock_guard<std::mutex> lk(h->mu);
    *out = tuning_of(h);
    return SSSP_OK;
}

int sssp_set_tuning(sssp_handle h, const sssp_tuning* t) {
    if (!h || !t || !valid_tuning(*t)) return SSSP_E_INVAL;
    DeviceGuard dg(h->device);
    std::lock_guard<std::mutex> lk(h->mu);
    return set_locked(h, *t);
}

int sssp_autotune(sssp_handle h, const uint32_t* sources, uint32_t nsrc, uint32_t reps,
                  sssp_tune_result* out) {
    if (!h || !sources || nsrc == 0) return SSSP_E_INVAL;
    for (u32 i = 0; i < nsrc; ++i)
        if (sources[i] >= h->n) return SSSP_E_SOURCE_RANGE;
    if (reps == 0) reps = 3;
    DeviceGuard dg(h->device);
    std::lock_guard<std::mutex> lk(h->mu);
    cudaStream_t st = h->stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        (void)cudaGetLastError();
        return SSSP_E_CUDA;
    }
    // One candidate: set it, one warm-up solve, then the best of `reps`
    // passes over the sources (device time of the whole pass).
    auto time = [&](const sssp_tuning& t, double* ms) -> int {
        RC(set_locked(h, t));
        Context& c = h->single;
        RC(enqueue_single(h, sources[0], 0, st, c.stage, nullptr, nullptr, nullptr, kNoTarget));
        double best = 1e30;
        for (u32 r = 0; r < reps; ++r) {
            CK(cudaEventRecord(e0, st));
            for (u32 i = 0; i < nsrc; ++i)
                RC(enqueue_single(h, sources[i], 0, st, c.stage, nullptr, nullptr, nullptr,
                                  kNoTarget));
            CK(cudaEventRecord(e1, st));
            CK(cudaEventSynchronize(e1));
            float f = 0;
            CK(cudaEventElapsedTime(&f, e0, e1));
            best = std::min(best, (double)f);
        }
        CK(cudaMemcpyAsync(c.h_ctl, c.P.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        if (c.h_ctl->error) return SSSP_E_INTERNAL;
        if (c.h_ctl->status == kErrRounds) return SSSP_E_ROUND_LIMIT;
        *ms = best;
        return SSSP_OK;
    };
    sssp_tune_result res{};
    int rc = sweep(tuning_of(h), time, &res);
    if (rc == SSSP_OK) rc = set_locked(h, res.best);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != SSSP_OK) return rc;
    char key[96];
    graph_key(h, key, sizeof(key));
    RC(sssp_tune_cache_put(key, &res.best));
    if (out) *out = res;
    return SSSP_OK;
}

int sssp_autotune_batch(const sssp_handle* g, const uint32_t* sources, uint32_t k, uint32_t reps,
                        sssp_tune_result* out) {
    if (!g || !sources || k == 0) return SSSP_E_INVAL;
    for (u32 i = 0; i < k; ++i) {
        if (!g[i]) return SSSP_E_INVAL;
        if (sources[i] >= g[i]->n) return SSSP_E_SOURCE_RANGE;
    }
    if (reps == 0) reps = 3;
    DeviceGuard dg(g[0]->device);
    // Device outputs for the timed batches: one array for every query.
    u64 total = 0;
    for (u32 i = 0; i < k; ++i) total += g[i]->n;
    u64* dist = nullptr;
    if (cudaMalloc(&dist, sizeof(u64) * total) != cudaSuccess) {
        (void)cudaGetLastError();
        return SSSP_E_NOMEM;
    }
    std::vector<u64*> outs(k);
    u64 off = 0;
    for (u32 i = 0; i < k; ++i) {
        outs[i] = dist + off;
        off += g[i]->n;
    }
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = SSSP_OK;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        (void)cudaGetLastError();
        rc = SSSP_E_CUDA;
    }
    auto time = [&](const sssp_tuning& t, double* ms) -> int {
        RC(batch_impl(g, sources, k, outs.data(), true, nullptr, st, true, &t));
        double best = 1e30;
        for (u32 r = 0; r < reps; ++r) {
            CK(cudaEventRecord(e0, st));
            RC(batch_impl(g, sources, k, outs.data(), true, nullptr, st, true, &t));
            CK(cudaEventRecord(e1, st));
            CK(cudaEventSynchronize(e1));
            float f = 0;
            CK(cudaEventElapsedTime(&f, e0, e1));
            best = std::min(best, (double)f);
        }
        *ms = best;
        return SSSP_OK;
    };
    sssp_tune_result res{};
    if (rc == SSSP_OK) {
        // Start from the batch's cached tuning, else the first handle's.
        sssp_tuning start = tuning_of(g[0]);
        char key[96];
        batch_key(g, k, key, sizeof(key));
        sssp_tuning cached{};
        if (tune_cache_find(key, &cached) == SSSP_OK) start = cached;
        rc = sweep(start, time, &res);
        if (rc == SSSP_OK) rc = sssp_tune_cache_put(key, &res.best);
    }
    if (st) cudaStreamSynchronize(st);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    cudaFree(dist);
    if (rc == SSSP_OK && out) *out = res;
    return rc;
}

}  // extern "C"
