/*
 * RASTER oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded CPU statement of what the RASTER hot path
 * computes, used to check the CUDA library.  Only the tests, the package's
 * smoke check and the benchmark's CPU-baseline leg may load it; the library
 * never does.  It shares no code, header or table with the CUDA path.
 *
 * It follows Alg. 1 (RASTER) of Ulm et al., "Contraction Clustering (RASTER)":
 *   contraction   -- project every point to its tile and count points per
 *                    tile (Alg. 1, first loop; Sect. 3.2), then drop tiles
 *                    with fewer than tau points (Alg. 1, second loop);
 *   agglomeration -- repeatedly pop a significant tile and collect every
 *                    significant tile reachable through neighbors(u, delta)
 *                    (Alg. 1, while loop): the tiles at Chebyshev or Manhattan
 *                    distance at most delta (Sect. 3.2; the paper's own
 *                    choice, and the default, is Chebyshev distance 1, the
 *                    eight neighbours), keeping clusters of at least mu tiles.
 * Points have two coordinates, or three (Sect. 3.6, "Generalizing to Higher
 * Dimensions": the same method on d-dimensional tiles, whose neighbours at
 * Chebyshev distance 1 are the 3^d - 1 surrounding tiles).
 * Optionally (Sect. 3.6, "disadvantageous grid layouts", Fig. 4) the
 * significant tiles also include every occupied tile of any group of 2 x 2
 * tiles that holds at least tau points together.
 * Points may arrive in any number of chunks ("Working with huge data sets",
 * Sect. 3.6); the counts only depend on the multiset of points.
 *
 * Readings where the paper leaves a choice open (each is a fixed convention
 * of this project, shared with the CUDA library by specification only):
 *   - projection: ix = floor(fl(x * s)) with s = 10^precision held as one
 *     double, fl() one IEEE-754 binary64 multiply rounded to nearest even
 *     (build with -ffp-contract=off so no fused multiply-add appears);
 *     floor, not truncation toward zero, so tiles are uniform across 0;
 *   - a tile index must lie in [INT32_MIN+1, INT32_MAX-1]; a non-finite or
 *     out-of-range coordinate is an error (ORACLE_RANGE) and that point is
 *     skipped;
 *   - key = (int64)ix << 32 | (uint32)iy;
 *   - three coordinates: each index must lie in [-(2^20 - 1), 2^20 - 2];
 *     key = (ix + 2^20) << 42 | (iy + 2^20) << 21 | (iz + 2^20), so integer
 *     order of keys is (ix, iy, iz) order;
 *   - significant: count >= tau; kept: cluster size (in tiles) >= mu;
 *   - cluster id = key of the cluster's smallest tile in (ix, iy)
 *     lexicographic order; noise label = INT64_MIN;
 *   - outputs are listed in (ix, iy) lexicographic order.
 */
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <unordered_map>
#include <unordered_set>
#include <vector>

namespace {

const int ORACLE_OK = 0;
const int ORACLE_RANGE = 2;
const int64_t NOISE = INT64_MIN;

struct Tile {
    int32_t ix, iy;
};

int64_t pack(int32_t ix, int32_t iy) {
    return (int64_t)(((uint64_t)(uint32_t)ix << 32) | (uint64_t)(uint32_t)iy);
}
int32_t tile_x(int64_t key) { return (int32_t)(uint32_t)((uint64_t)key >> 32); }
int32_t tile_y(int64_t key) { return (int32_t)(uint32_t)((uint64_t)key & 0xffffffffu); }

/* (ix, iy) lexicographic order on keys. */
bool tile_less(int64_t a, int64_t b) {
    if (tile_x(a) != tile_x(b)) return tile_x(a) < tile_x(b);
    return tile_y(a) < tile_y(b);
}

/* project(x, y, prec) of Alg. 1: one coordinate.  Returns false when the
 * scaled coordinate is not finite or its floor leaves the valid range. */
bool project_coord(double v, double scale, int32_t *out) {
    volatile double scaled = v * scale;  /* one rounded multiply */
    double f = std::floor(scaled);
    if (!(f >= -2147483647.0 && f <= 2147483646.0)) return false;  /* also rejects NaN */
    *out = (int32_t)f;
    return true;
}

bool project(double x, double y, double scale, int64_t *key) {
    int32_t ix, iy;
    if (!project_coord(x, scale, &ix) || !project_coord(y, scale, &iy)) return false;
    *key = pack(ix, iy);
    return true;
}

/* Three coordinates: 21-bit fields, each index offset by 2^20. */
const int64_t BIAS3 = (int64_t)1 << 20;
const int64_t MIN3 = -(BIAS3 - 1), MAX3 = BIAS3 - 2;

int64_t pack3(int64_t ix, int64_t iy, int64_t iz) {
    return ((ix + BIAS3) << 42) | ((iy + BIAS3) << 21) | (iz + BIAS3);
}
int64_t tile3(int64_t key, int axis) { return ((key >> (42 - 21 * axis)) & 0x1FFFFF) - BIAS3; }

bool project_coord3(double v, double scale, int64_t *out) {
    volatile double product = scale * v; /* one rounded multiply */
    double f = std::floor(product);
    if (!(f >= (double)MIN3 && f <= (double)MAX3)) return false;
    *out = (int64_t)f;
    return true;
}

/* Project point i of an array of `dims` coordinates per point. */
bool project_point(const double *xy, int64_t i, int dims, double scale, int64_t *key) {
    if (dims == 3) {
        int64_t c[3];
        for (int a = 0; a < 3; ++a)
            if (!project_coord3(xy[3 * i + a], scale, &c[a])) return false;
        *key = pack3(c[0], c[1], c[2]);
        return true;
    }
    return project(xy[2 * i], xy[2 * i + 1], scale, key);
}

/* The tile at offset (dx, dy, dz) from u, if its indices are valid. */
bool neighbour_key(int64_t u, int dx, int dy, int dz, int dims, int64_t *out) {
    if (dims == 3) {
        const int64_t n[3] = {tile3(u, 0) + dx, tile3(u, 1) + dy, tile3(u, 2) + dz};
        for (int a = 0; a < 3; ++a)
            if (n[a] < MIN3 || n[a] > MAX3) return false;
        *out = pack3(n[0], n[1], n[2]);
        return true;
    }
    /* tiles outside the valid index range never exist */
    int64_t nx = (int64_t)tile_x(u) + dx, ny = (int64_t)tile_y(u) + dy;
    if (nx < -2147483647LL || nx > 2147483646LL) return false;
    if (ny < -2147483647LL || ny > 2147483646LL) return false;
    *out = pack((int32_t)nx, (int32_t)ny);
    return true;
}

}  // namespace

const int ORACLE_CHEBYSHEV = 0;
const int ORACLE_MANHATTAN = 1;

struct oracle_state {
    double scale;
    uint32_t tau, mu;
    int metric;    /* ORACLE_CHEBYSHEV or ORACLE_MANHATTAN */
    int delta;     /* neighbourhood radius in tiles */
    int groups;    /* 1: 2 x 2 groups of Sect. 3.6 also make tiles significant */
    int dims;      /* coordinates per point: 2 or 3 */
    int status;
    int64_t points;
    /* acc of Alg. 1: tile -> number of points */
    std::unordered_map<int64_t, uint64_t> acc;
    /* agglomeration results */
    bool finished;
    int64_t n_significant;
    std::vector<int64_t> kept_key;
    std::vector<uint64_t> kept_count;
    std::vector<int64_t> kept_cid;
    int64_t n_clusters;
    std::unordered_map<int64_t, int64_t> cid_of;  /* kept tile -> cluster id */
};

/* (ix, iy[, iz]) lexicographic order of two keys. */
static bool before(const oracle_state *s, int64_t a, int64_t b) { return s->dims == 3 ? a < b : tile_less(a, b); }

extern "C" {

oracle_state *oracle_create_ex(double scale, uint32_t tau, uint32_t mu, int metric, int delta, int groups,
                               int dims) {
    oracle_state *s = new oracle_state();
    s->scale = scale;
    s->tau = tau;
    s->mu = mu;
    s->metric = metric;
    s->delta = delta;
    s->groups = groups;
    s->dims = dims;
    s->status = ORACLE_OK;
    s->points = 0;
    s->finished = false;
    s->n_significant = 0;
    s->n_clusters = 0;
    return s;
}

oracle_state *oracle_create(double scale, uint32_t tau, uint32_t mu) {
    return oracle_create_ex(scale, tau, mu, ORACLE_CHEBYSHEV, 1, 0, 2);
}

void oracle_free(oracle_state *s) { delete s; }

/* Contraction for one chunk of points (Alg. 1, first loop). */
int oracle_add(oracle_state *s, const double *xy, int64_t n) {
    for (int64_t i = 0; i < n; ++i) {
        int64_t key;
        if (!project_point(xy, i, s->dims, s->scale, &key)) {
            s->status = ORACLE_RANGE;
            continue;
        }
        auto it = s->acc.find(key);
        if (it == s->acc.end())
            s->acc[key] = 1;
        else
            it->second += 1;
        s->points += 1;
    }
    s->finished = false;
    return s->status;
}

/* Threshold and agglomeration (Alg. 1, second loop and while loop). */
int oracle_finish(oracle_state *s) {
    /* second loop: keep the tiles with at least tau points */
    std::unordered_set<int64_t> sigma;
    for (const auto &kv : s->acc)
        if (kv.second >= s->tau) sigma.insert(kv.first);
    /* Sect. 3.6: an occupied tile is also kept when one of the four 2 x 2
     * groups it belongs to holds at least tau points in total */
    if (s->groups && s->dims == 2) {
        for (const auto &kv : s->acc) {
            const int64_t x = tile_x(kv.first), y = tile_y(kv.first);
            bool keep = false;
            for (int ax = -1; ax <= 0 && !keep; ++ax)
                for (int ay = -1; ay <= 0 && !keep; ++ay) {
                    uint64_t total = 0;
                    for (int gx = 0; gx <= 1; ++gx)
                        for (int gy = 0; gy <= 1; ++gy) {
                            const int64_t tx = x + ax + gx, ty = y + ay + gy;
                            if (tx < -2147483647LL || tx > 2147483646LL) continue;
                            if (ty < -2147483647LL || ty > 2147483646LL) continue;
                            auto it = s->acc.find(pack((int32_t)tx, (int32_t)ty));
                            if (it != s->acc.end()) total += it->second;
                        }
                    if (total >= s->tau) keep = true;
                }
            if (keep) sigma.insert(kv.first);
        }
    }
    s->n_significant = (int64_t)sigma.size();

    s->kept_key.clear();
    s->kept_count.clear();
    s->kept_cid.clear();
    s->cid_of.clear();
    s->n_clusters = 0;

    /* while loop: pop a tile, gather its cluster by visiting neighbours */
    std::vector<std::vector<int64_t>> clusters;
    while (!sigma.empty()) {
        int64_t t = *sigma.begin();
        sigma.erase(sigma.begin());
        std::vector<int64_t> cluster;
        std::deque<int64_t> visit;
        visit.push_back(t);
        while (!visit.empty()) {
            int64_t u = visit.front();
            visit.pop_front();
            std::vector<int64_t> ns;  /* neighbors(u, delta) in sigma */
            const int dz_max = s->dims == 3 ? s->delta : 0;
            for (int dx = -s->delta; dx <= s->delta; ++dx)
                for (int dy = -s->delta; dy <= s->delta; ++dy)
                    for (int dz = -dz_max; dz <= dz_max; ++dz) {
                        if (dx == 0 && dy == 0 && dz == 0) continue;
                        if (s->metric == ORACLE_MANHATTAN && std::abs(dx) + std::abs(dy) + std::abs(dz) > s->delta)
                            continue;
                        int64_t nk;
                        if (!neighbour_key(u, dx, dy, dz, s->dims, &nk)) continue;
                        if (sigma.count(nk)) ns.push_back(nk);
                    }
            cluster.push_back(u);
            for (int64_t k : ns) {
                sigma.erase(k);
                visit.push_back(k);
            }
        }
        if (cluster.size() >= s->mu) clusters.push_back(cluster);
    }

    /* emit kept tiles with their cluster id = smallest tile of the cluster */
    std::vector<std::pair<int64_t, int64_t>> rows;  /* (key, cid) */
    for (const auto &c : clusters) {
        int64_t cid = c[0];
        for (int64_t k : c)
            if (before(s, k, cid)) cid = k;
        for (int64_t k : c) rows.push_back({k, cid});
        s->cid_of.reserve(s->cid_of.size() + c.size());
        for (int64_t k : c) s->cid_of[k] = cid;
    }
    std::sort(rows.begin(), rows.end(),
              [s](const std::pair<int64_t, int64_t> &a, const std::pair<int64_t, int64_t> &b) {
                  return before(s, a.first, b.first);
              });
    for (const auto &r : rows) {
        s->kept_key.push_back(r.first);
        s->kept_count.push_back(s->acc[r.first]);
        s->kept_cid.push_back(r.second);
    }
    s->n_clusters = (int64_t)clusters.size();
    s->finished = true;
    return s->status;
}

int oracle_status(const oracle_state *s) { return s->status; }
int64_t oracle_points(const oracle_state *s) { return s->points; }
int64_t oracle_n_tiles(const oracle_state *s) { return (int64_t)s->acc.size(); }
int64_t oracle_n_significant(const oracle_state *s) { return s->n_significant; }
int64_t oracle_n_kept(const oracle_state *s) { return (int64_t)s->kept_key.size(); }
int64_t oracle_n_clusters(const oracle_state *s) { return s->n_clusters; }

/* All tiles with their counts, in (ix, iy) order. */
void oracle_copy_tiles(const oracle_state *s, int64_t *key, uint64_t *count) {
    std::vector<int64_t> keys;
    keys.reserve(s->acc.size());
    for (const auto &kv : s->acc) keys.push_back(kv.first);
    std::sort(keys.begin(), keys.end(), [s](int64_t a, int64_t b) { return before(s, a, b); });
    for (size_t i = 0; i < keys.size(); ++i) {
        key[i] = keys[i];
        count[i] = s->acc.at(keys[i]);
    }
}

/* Tiles of kept clusters with (count, cluster id), in (ix, iy) order. */
void oracle_copy_kept(const oracle_state *s, int64_t *key, uint64_t *count, int64_t *cid) {
    for (size_t i = 0; i < s->kept_key.size(); ++i) {
        key[i] = s->kept_key[i];
        count[i] = s->kept_count[i];
        cid[i] = s->kept_cid[i];
    }
}

/* Per-point labels: the RASTER* second pass (Sect. 4.1, Experiment 1) that
 * projects every point again and reports its tile's cluster, or noise.
 * Returns ORACLE_RANGE if some point could not be projected (it gets noise). */
int oracle_labels(const oracle_state *s, const double *xy, int64_t n, int64_t *labels) {
    int st = ORACLE_OK;
    for (int64_t i = 0; i < n; ++i) {
        int64_t key;
        if (!project_point(xy, i, s->dims, s->scale, &key)) {
            labels[i] = NOISE;
            st = ORACLE_RANGE;
            continue;
        }
        auto it = s->cid_of.find(key);
        labels[i] = (it == s->cid_of.end()) ? NOISE : it->second;
    }
    return st;
}

/* RASTER' output (Sect. 3.4): the points of every kept tile, rows in the
 * order of oracle_copy_kept, indices increasing within a row.  row_start has
 * n_kept + 1 entries; idx has room for `capacity` indices.  Returns the number
 * of grouped points (idx untouched if it exceeds capacity). */
int64_t oracle_point_groups(const oracle_state *s, const double *xy, int64_t n, int64_t *row_start, int64_t *idx,
                            int64_t capacity) {
    std::unordered_map<int64_t, int64_t> row_of;
    for (size_t r = 0; r < s->kept_key.size(); ++r) row_of[s->kept_key[r]] = (int64_t)r;
    std::vector<int64_t> rows(n, -1), count(s->kept_key.size(), 0);
    for (int64_t i = 0; i < n; ++i) {
        int64_t key;
        if (!project_point(xy, i, s->dims, s->scale, &key)) continue;
        auto it = row_of.find(key);
        if (it == row_of.end()) continue;
        rows[i] = it->second;
        count[it->second] += 1;
    }
    row_start[0] = 0;
    for (size_t r = 0; r < count.size(); ++r) row_start[r + 1] = row_start[r] + count[r];
    const int64_t m = row_start[count.size()];
    if (m > capacity) return m;
    std::vector<int64_t> cursor(row_start, row_start + count.size());
    for (int64_t i = 0; i < n; ++i)
        if (rows[i] >= 0) idx[cursor[rows[i]]++] = i;
    return m;
}

/* Projection alone, for pinning: keys[i] and ok[i] (1 valid, 0 range error). */
void oracle_project(const double *xy, int64_t n, double scale, int64_t *keys, uint8_t *ok, int dims) {
    for (int64_t i = 0; i < n; ++i) {
        int64_t key = 0;
        bool good = project_point(xy, i, dims, scale, &key);
        keys[i] = good ? key : 0;
        ok[i] = good ? 1 : 0;
    }
}

/* Exact counts of a given set of tiles over a point set (one pass), used to
 * check sampled outputs of very large runs one by one.  counts[j] is the
 * number of points whose tile is keys[j]; a key may be queried more than
 * once, and points with a range error count nowhere. */
void oracle_count_keys(const double *xy, int64_t n, double scale, const int64_t *keys, int64_t k,
                       uint64_t *counts, int dims) {
    std::unordered_map<int64_t, uint64_t> tally;
    for (int64_t j = 0; j < k; ++j) tally[keys[j]] = 0;
    for (int64_t i = 0; i < n; ++i) {
        int64_t key;
        if (!project_point(xy, i, dims, scale, &key)) continue;
        auto it = tally.find(key);
        if (it != tally.end()) it->second += 1;
    }
    for (int64_t j = 0; j < k; ++j) counts[j] = tally.at(keys[j]);
}

}  // extern "C"
