/*
 * P-RASTER on the host cores -- TEST AND BENCHMARK INFRASTRUCTURE ONLY.
 *
 * The multi-threaded CPU form of RASTER that the paper describes in Sect. 3.5
 * (P-RASTER; Alg. 2 and Alg. 3; correctness in App. C), used as the timed
 * multi-core CPU baseline beside the single-threaded oracle.  It shares no
 * code with the CUDA library.  Steps, in the paper's order:
 *   1. contraction: the input is cut into unsorted batches, one per thread;
 *      each thread projects its points and counts them in its own hash map;
 *   2. join: the per-thread maps are joined (here in parallel: thread t joins
 *      the keys whose hash falls in its share, where the paper's code joined
 *      sequentially), then tiles with fewer than tau points are dropped;
 *   3. agglomeration (Alg. 2): the significant tiles are sorted into N
 *      vertical slices by their x index; each slice is clustered in parallel
 *      (8-neighbour search within the slice); clusters touching no border are
 *      kept if they have at least mu tiles, the others become candidates;
 *   4. joining (Alg. 3): borders are processed from right to left; the
 *      candidates touching border B_i are merged through their neighbouring
 *      tiles; a merged cluster that also touches B_(i-1) is carried on to the
 *      next border, otherwise it is kept if it has at least mu tiles;
 *   5. labels (RASTER*, Sect. 4.1): a parallel pass projects every point again
 *      and reports its tile's cluster id.
 * Conventions are those of the oracle: floor(fl(x * s)) with -ffp-contract=off,
 * indices in [INT32_MIN+1, INT32_MAX-1], key = ix << 32 | (uint32)iy,
 * cluster id = (ix, iy)-smallest tile, noise = INT64_MIN.  Two coordinates,
 * Chebyshev distance 1 (the paper's choice).
 */
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdint>
#include <deque>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

namespace {

const int64_t NOISE = INT64_MIN;

int64_t pack(int32_t ix, int32_t iy) { return (int64_t)(((uint64_t)(uint32_t)ix << 32) | (uint64_t)(uint32_t)iy); }
int32_t tx(int64_t k) { return (int32_t)(uint32_t)((uint64_t)k >> 32); }
int32_t ty(int64_t k) { return (int32_t)(uint32_t)((uint64_t)k & 0xffffffffu); }
bool lexless(int64_t a, int64_t b) { return tx(a) != tx(b) ? tx(a) < tx(b) : ty(a) < ty(b); }

bool coord(double v, double s, int32_t *out) {
    volatile double p = v * s;
    const double f = std::floor(p);
    if (!(f >= -2147483647.0 && f <= 2147483646.0)) return false;
    *out = (int32_t)f;
    return true;
}

bool project(const double *xy, int64_t i, double s, int64_t *key) {
    int32_t a, b;
    if (!coord(xy[2 * i], s, &a) || !coord(xy[2 * i + 1], s, &b)) return false;
    *key = pack(a, b);
    return true;
}

uint64_t mix(int64_t k) {
    uint64_t z = (uint64_t)k + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

template <typename F>
void parallel(int threads, F f) {
    std::vector<std::thread> th;
    for (int t = 1; t < threads; ++t) th.emplace_back(f, t);
    f(0);
    for (auto &x : th) x.join();
}

double now() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// Open-addressing hash map from tile key to a 64-bit value (linear probing,
// at most half full; the unreachable key INT64_MIN marks an empty slot).  A
// flat table keeps every thread's inserts free of the allocator.
class FlatMap {
public:
    explicit FlatMap(size_t expect = 16) { rehash(capacity_for(expect)); }
    uint64_t &get(int64_t k) {  // the value of k, inserted as 0 if absent
        if ((n_ + 1) * 2 > keys_.size()) rehash(keys_.size() * 2);
        size_t i = home(k);
        while (keys_[i] != kEmpty && keys_[i] != k) i = (i + 1) & mask_;
        if (keys_[i] == kEmpty) {
            keys_[i] = k;
            vals_[i] = 0;
            ++n_;
        }
        return vals_[i];
    }
    const uint64_t *find(int64_t k) const {
        size_t i = home(k);
        while (keys_[i] != kEmpty) {
            if (keys_[i] == k) return &vals_[i];
            i = (i + 1) & mask_;
        }
        return nullptr;
    }
    size_t size() const { return n_; }
    template <typename F>
    void each(F f) const {
        for (size_t i = 0; i < keys_.size(); ++i)
            if (keys_[i] != kEmpty) f(keys_[i], vals_[i]);
    }
    void release() {
        std::vector<int64_t>().swap(keys_);
        std::vector<uint64_t>().swap(vals_);
        n_ = 0;
    }

private:
    static constexpr int64_t kEmpty = INT64_MIN;
    static size_t capacity_for(size_t expect) {
        size_t c = 16;
        while (c < 2 * expect + 2) c <<= 1;
        return c;
    }
    size_t home(int64_t k) const { return (size_t)(mix(k) >> shift_); }  // high bits: shares use the low ones
    void rehash(size_t cap) {
        std::vector<int64_t> ok;
        std::vector<uint64_t> ov;
        ok.swap(keys_);
        ov.swap(vals_);
        keys_.assign(cap, kEmpty);
        vals_.assign(cap, 0);
        mask_ = cap - 1;
        shift_ = 64;
        for (size_t c = cap; c > 1; c >>= 1) --shift_;
        n_ = 0;
        for (size_t i = 0; i < ok.size(); ++i)
            if (ok[i] != kEmpty) get(ok[i]) = ov[i];
    }
    std::vector<int64_t> keys_;
    std::vector<uint64_t> vals_;
    size_t mask_ = 0, n_ = 0;
    int shift_ = 64;
};

struct Cluster {
    std::vector<int64_t> tiles;
    bool left = false, right = false;  // touches the slice's left / right border
};

}  // namespace

struct praster_state {
    double scale;
    uint32_t tau, mu;
    int threads;
    int status;
    int64_t n_tiles, n_significant, n_clusters;
    std::vector<int64_t> key, cid;
    std::vector<uint64_t> count;
    std::vector<FlatMap> cid_of;  // per key share: kept tile -> cluster id (as uint64)
    double t_contract, t_agglomerate, t_labels;
};

extern "C" {

praster_state *praster_create(double scale, uint32_t tau, uint32_t mu, int threads) {
    praster_state *s = new praster_state();
    s->scale = scale;
    s->tau = tau;
    s->mu = mu;
    s->threads = std::max(1, threads);
    s->status = 0;
    s->n_tiles = s->n_significant = s->n_clusters = 0;
    s->t_contract = s->t_agglomerate = s->t_labels = 0;
    return s;
}

void praster_free(praster_state *s) { delete s; }

/* Steps 1-4 over the n points (one batch of the whole input). */
int praster_run(praster_state *s, const double *xy, int64_t n) {
    const int T = s->threads;
    const double t0 = now();
    // 1. per-thread hash maps over unsorted batches; each thread keeps one map
    // per share of the key space, so that the join reads only its own share
    std::vector<std::vector<FlatMap>> local(T);
    std::vector<int> bad(T, 0);
    parallel(T, [&](int t) {
        const int64_t lo = n * t / T, hi = n * (t + 1) / T;
        auto &m = local[t];
        m.assign(T, FlatMap((size_t)((hi - lo) / (2 * T) + 16)));
        for (int64_t i = lo; i < hi; ++i) {
            int64_t k;
            if (!project(xy, i, s->scale, &k)) {
                bad[t] = 1;
                continue;
            }
            m[(int)(mix(k) % (uint64_t)T)].get(k) += 1;
        }
    });
    // 2. join: thread t joins share t of every thread's maps (the paper's code
    // joined the maps sequentially)
    std::vector<FlatMap> joined(T);
    parallel(T, [&](int t) {
        size_t guess = 0;
        for (auto &l : local) guess = std::max(guess, l[t].size());
        FlatMap m(guess + guess / 2 + 16);
        for (auto &l : local) {
            l[t].each([&](int64_t k, uint64_t v) { m.get(k) += v; });
            l[t].release();
        }
        joined[t] = std::move(m);
    });
    local.clear();
    s->status = *std::max_element(bad.begin(), bad.end()) ? 2 : 0;
    const double t1 = now();
    s->t_contract = t1 - t0;

    // significant tiles, and the tile count
    std::vector<std::vector<int64_t>> sig_part(T);
    int64_t tiles = 0;
    for (auto &m : joined) tiles += (int64_t)m.size();
    parallel(T, [&](int t) {
        joined[t].each([&](int64_t k, uint64_t v) {
            if (v >= s->tau) sig_part[t].push_back(k);
        });
    });
    std::vector<int64_t> sig;
    for (auto &p : sig_part) sig.insert(sig.end(), p.begin(), p.end());
    s->n_tiles = tiles;
    s->n_significant = (int64_t)sig.size();

    // 3. Alg. 2: N vertical slices of equal width in x
    const int N = T;
    int64_t xmin = INT64_MAX, xmax = INT64_MIN;
    for (int64_t k : sig) {
        xmin = std::min<int64_t>(xmin, tx(k));
        xmax = std::max<int64_t>(xmax, tx(k));
    }
    const int64_t width = sig.empty() ? 1 : (xmax - xmin) / N + 1;
    auto slice_of = [&](int64_t k) { return (int)std::min<int64_t>(N - 1, (tx(k) - xmin) / width); };
    auto lo_x = [&](int sl) { return xmin + (int64_t)sl * width; };
    auto hi_x = [&](int sl) { return sl == N - 1 ? xmax : xmin + (int64_t)(sl + 1) * width - 1; };
    std::vector<std::vector<int64_t>> slice(N);
    for (int64_t k : sig) slice[slice_of(k)].push_back(k);
    std::vector<std::vector<Cluster>> kept(N), cand(N);
    parallel(N, [&](int sl) {
        // the slice's tiles; value 1 while not yet visited
        FlatMap rest(slice[sl].size());
        for (int64_t k : slice[sl]) rest.get(k) = 1;
        const int64_t x0 = lo_x(sl), x1 = hi_x(sl);
        std::vector<int64_t> visit;
        for (int64_t start : slice[sl]) {
            uint64_t &st = rest.get(start);
            if (!st) continue;
            st = 0;
            Cluster c;
            visit.assign(1, start);
            for (size_t q = 0; q < visit.size(); ++q) {
                const int64_t u = visit[q];
                c.tiles.push_back(u);
                if (sl > 0 && tx(u) == x0) c.left = true;
                if (sl < N - 1 && tx(u) == x1) c.right = true;
                for (int dx = -1; dx <= 1; ++dx)
                    for (int dy = -1; dy <= 1; ++dy) {
                        if (!dx && !dy) continue;
                        const int64_t nx = (int64_t)tx(u) + dx, ny = (int64_t)ty(u) + dy;
                        if (nx < -2147483647LL || nx > 2147483646LL || ny < -2147483647LL || ny > 2147483646LL)
                            continue;
                        const int64_t nk = pack((int32_t)nx, (int32_t)ny);
                        const uint64_t *f = rest.find(nk);
                        if (f && *f) {
                            rest.get(nk) = 0;
                            visit.push_back(nk);
                        }
                    }
            }
            if (c.left || c.right)
                cand[sl].push_back(std::move(c));
            else if (c.tiles.size() >= s->mu)
                kept[sl].push_back(std::move(c));
        }
    });
    // 4. Alg. 3: join across borders B_(N-1) .. B_1, right to left.  Border
    // B_i lies between slices i-1 and i.  `carry` holds merged clusters that
    // reach further left (C_inter).
    std::vector<Cluster> out;
    for (auto &v : kept)
        for (auto &c : v) out.push_back(std::move(c));
    std::vector<Cluster> carry;
    for (int b = N - 1; b >= 1; --b) {
        // C_lr: candidates of slice b touching B_b (its left border), the
        // carried clusters (they touch B_b by construction), and candidates of
        // slice b-1 touching B_b (their right border)
        std::vector<Cluster> lr;
        std::vector<Cluster> keep_b;
        for (auto &c : cand[b]) {
            if (c.left)
                lr.push_back(std::move(c));
        }
        cand[b].clear();
        for (auto &c : carry) lr.push_back(std::move(c));
        carry.clear();
        for (auto &c : cand[b - 1]) {
            if (c.right)
                lr.push_back(std::move(c));
            else
                keep_b.push_back(std::move(c));
        }
        cand[b - 1] = std::move(keep_b);
        // tiles of the two border columns -> candidate
        const int64_t xl = hi_x(b - 1), xr = lo_x(b);
        std::unordered_map<int64_t, int> owner;
        for (int c = 0; c < (int)lr.size(); ++c)
            for (int64_t k : lr[c].tiles)
                if (tx(k) == xl || tx(k) == xr) owner[k] = c;
        std::vector<char> seen(lr.size(), 0);
        for (int c0 = 0; c0 < (int)lr.size(); ++c0) {
            if (seen[c0]) continue;
            seen[c0] = 1;
            Cluster j;
            std::vector<int> todo{c0};
            bool touches_left = false;
            for (size_t q = 0; q < todo.size(); ++q) {
                Cluster &v = lr[todo[q]];
                for (int64_t k : v.tiles) {
                    if (b - 1 > 0 && tx(k) == lo_x(b - 1) && slice_of(k) == b - 1) touches_left = true;
                    if (tx(k) != xl && tx(k) != xr) continue;
                    const int dx = tx(k) == xl ? 1 : -1;  // across the border
                    for (int dy = -1; dy <= 1; ++dy) {
                        const int64_t ny = (int64_t)ty(k) + dy;
                        if (ny < -2147483647LL || ny > 2147483646LL) continue;
                        auto it = owner.find(pack(tx(k) + dx, (int32_t)ny));
                        if (it != owner.end() && !seen[it->second]) {
                            seen[it->second] = 1;
                            todo.push_back(it->second);
                        }
                    }
                }
                j.tiles.insert(j.tiles.end(), v.tiles.begin(), v.tiles.end());
                touches_left = touches_left || (v.left && slice_of(v.tiles[0]) == b - 1);
            }
            if (touches_left) {
                j.left = true;
                carry.push_back(std::move(j));
            } else if (j.tiles.size() >= s->mu) {
                out.push_back(std::move(j));
            }
        }
    }
    // candidates left in slice 0 cannot touch a border any more
    for (auto &c : cand[0])
        if (c.tiles.size() >= s->mu) out.push_back(std::move(c));
    for (auto &c : carry)
        if (c.tiles.size() >= s->mu) out.push_back(std::move(c));

    // rows with cluster ids, cluster by cluster (the caller sorts them when it
    // needs an order); ids, counts and the label map are filled in parallel
    std::vector<size_t> first(out.size() + 1, 0);
    for (size_t c = 0; c < out.size(); ++c) first[c + 1] = first[c] + out[c].tiles.size();
    const size_t R = first.back();
    s->key.resize(R);
    s->cid.resize(R);
    s->count.resize(R);
    parallel(T, [&](int t) {
        for (size_t c = out.size() * t / T; c < out.size() * (t + 1) / T; ++c) {
            int64_t id = out[c].tiles[0];
            for (int64_t k : out[c].tiles)
                if (lexless(k, id)) id = k;
            size_t r = first[c];
            for (int64_t k : out[c].tiles) {
                s->key[r] = k;
                s->cid[r] = id;
                s->count[r] = *joined[(int)(mix(k) % (uint64_t)T)].find(k);
                ++r;
            }
        }
    });
    // label map: thread t holds the kept tiles of its key share
    s->cid_of.assign(T, FlatMap());
    parallel(T, [&](int t) {
        FlatMap m(R / T + 16);
        for (size_t r = 0; r < R; ++r)
            if ((int)(mix(s->key[r]) % (uint64_t)T) == t) m.get(s->key[r]) = (uint64_t)s->cid[r];
        s->cid_of[t] = std::move(m);
    });
    s->n_clusters = (int64_t)out.size();
    s->t_agglomerate = now() - t1;
    return s->status;
}

/* Step 5: labels of n points, in parallel. */
int praster_labels(praster_state *s, const double *xy, int64_t n, int64_t *labels) {
    const double t0 = now();
    const int T = s->threads;
    std::vector<int> bad(T, 0);
    parallel(T, [&](int t) {
        for (int64_t i = n * t / T; i < n * (t + 1) / T; ++i) {
            int64_t k;
            if (!project(xy, i, s->scale, &k)) {
                labels[i] = NOISE;
                bad[t] = 1;
                continue;
            }
            const uint64_t *c = s->cid_of[(int)(mix(k) % (uint64_t)T)].find(k);
            labels[i] = c ? (int64_t)*c : NOISE;
        }
    });
    s->t_labels = now() - t0;
    return *std::max_element(bad.begin(), bad.end()) ? 2 : 0;
}

int64_t praster_n_tiles(const praster_state *s) { return s->n_tiles; }
int64_t praster_n_significant(const praster_state *s) { return s->n_significant; }
int64_t praster_n_clusters(const praster_state *s) { return s->n_clusters; }
int64_t praster_n_kept(const praster_state *s) { return (int64_t)s->key.size(); }

void praster_copy_kept(const praster_state *s, int64_t *key, uint64_t *count, int64_t *cid) {
    for (size_t i = 0; i < s->key.size(); ++i) {
        key[i] = s->key[i];
        count[i] = s->count[i];
        cid[i] = s->cid[i];
    }
}

/* Seconds of the last run: contraction (steps 1-2), agglomeration (3-4), labels (5). */
void praster_times(const praster_state *s, double *out) {
    out[0] = s->t_contract;
    out[1] = s->t_agglomerate;
    out[2] = s->t_labels;
}

}  // extern "C"
