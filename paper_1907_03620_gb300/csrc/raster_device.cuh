// Device building blocks of the RASTER hot path on sm_103a.
//
//   * project  -- the tile of a coordinate, floor(RN(v * s)) (Alg. 1
//                 project(), Sect. 3.2), evaluated exactly in 64-bit integer
//                 arithmetic.  GB300's FP64 pipe runs at ~1/64 of the integer
//                 rate, so the IEEE product is rebuilt from the significands:
//                 the exact product of v's 53-bit significand with the odd
//                 part of s's significand, rounded once to 53 significant bits
//                 (ties to even), then floored by shifting.  Zeros are exact;
//                 only non-finite/subnormal inputs and subnormal products take
//                 the FP64 instructions (__dmul_rn then floor).
//   * tile table -- open addressing with linear probing over 16-byte slots
//                 {key, count, aux}; key EMPTY = INT64_MIN is unreachable
//                 because ix = INT32_MIN is not a valid tile index.
//   * union-find -- hooking of the larger index under the smaller with
//                 atomicCAS and path halving (connected components of the
//                 significant tiles, Alg. 1 while loop).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "raster_project.cuh"

namespace raster {

constexpr unsigned long long kEmptyKey = 0x8000000000000000ull;
constexpr unsigned long long kInvalidKey = 0x8000000000000001ull;  // a point that did not project
constexpr unsigned int kAuxNone = 0xFFFFFFFFu;
// Marks a tile made significant by a 2 x 2 group (between the group pass and
// the selection of significant tiles only).
constexpr unsigned int kAuxGroup = 0xFFFFFFFEu;

// Status bits accumulated on the device (mapped to RASTER_E_* by the host).
constexpr unsigned int kStRange = 1u;
constexpr unsigned int kStFull = 2u;
constexpr unsigned int kStInternal = 4u;

struct __align__(16) Slot {
    unsigned long long key;
    unsigned int count;
    unsigned int aux;  // significant index during agglomeration, then label code
};

__device__ __forceinline__ unsigned long long pack_key(int ix, int iy) {
    return ((unsigned long long)(unsigned int)ix << 32) | (unsigned long long)(unsigned int)iy;
}
__device__ __forceinline__ int key_x(unsigned long long k) { return (int)(unsigned int)(k >> 32); }
__device__ __forceinline__ int key_y(unsigned long long k) { return (int)(unsigned int)k; }

// (ix, iy) lexicographic order as an unsigned 64-bit value.
__device__ __forceinline__ unsigned long long order_of(unsigned long long k) {
    return k ^ 0x8000000080000000ull;
}
__device__ __forceinline__ unsigned long long key_of_order(unsigned long long o) {
    return o ^ 0x8000000080000000ull;
}

// Three coordinates (the generalisation of Sect. 3.6 to higher dimensions):
// each index in [-(2^20 - 1), 2^20 - 2], stored plus 2^20 in a 21-bit field,
// x in the top field, so that integer key order is (x, y, z) order and the top
// bit is clear (no key equals kEmptyKey or kInvalidKey).
constexpr long long kBias3 = 1ll << 20;
constexpr int kMin3 = -(int)(kBias3 - 1), kMax3 = (int)(kBias3 - 2);
__device__ __forceinline__ unsigned long long pack_key3(long long ix, long long iy, long long iz) {
    return ((unsigned long long)(ix + kBias3) << 42) | ((unsigned long long)(iy + kBias3) << 21) |
           (unsigned long long)(iz + kBias3);
}
__device__ __forceinline__ int key3(unsigned long long k, int axis) {
    return (int)((k >> (42 - 21 * axis)) & 0x1FFFFFull) - (int)kBias3;
}

template <bool WIDE>
__device__ __forceinline__ unsigned long long project_point3(double x, double y, double z, const ProjParams& pp) {
    int ix, iy, iz;
    const bool ok = project_coord<WIDE>(x, pp, &ix) & project_coord<WIDE>(y, pp, &iy) & project_coord<WIDE>(z, pp, &iz);
    if (!ok || ix < kMin3 || ix > kMax3 || iy < kMin3 || iy > kMax3 || iz < kMin3 || iz > kMax3) return kInvalidKey;
    return pack_key3(ix, iy, iz);
}

template <bool WIDE>
__device__ __forceinline__ unsigned long long project_point(double x, double y, const ProjParams& pp) {
    int ix, iy;
    const bool okx = project_coord<WIDE>(x, pp, &ix);
    const bool oky = project_coord<WIDE>(y, pp, &iy);
    return (okx && oky) ? pack_key(ix, iy) : kInvalidKey;
}

// 32-bit tile hash: multiplicative combine of (ix, iy), then the MurmurHash3
// 32-bit finaliser (Appleby, public domain) for avalanche.
__device__ __forceinline__ unsigned int tile_hash(unsigned long long key) {
    unsigned int h = (unsigned int)(key >> 32) * 0x9E3779B1u + (unsigned int)key;
    h ^= h >> 16;
    h *= 0x85EBCA6Bu;
    h ^= h >> 13;
    h *= 0xC2B2AE35u;
    h ^= h >> 16;
    return h;
}

__device__ __forceinline__ unsigned long long load_key(const Slot* s) {
    return *reinterpret_cast<const volatile unsigned long long*>(&s->key);
}

// Add c points to tile `key`.  Returns 1 if the key was new, 0 if it existed,
// -1 if max_probe slots were probed without success (table full).
__device__ __forceinline__ int table_add(Slot* tab, unsigned int mask, unsigned long long key, unsigned int c,
                                         unsigned int max_probe) {
    unsigned int i = tile_hash(key) & mask;
    for (unsigned int p = 0; p < max_probe; ++p) {
        unsigned long long k = load_key(&tab[i]);
        if (k == key) {
            atomicAdd(&tab[i].count, c);
            return 0;
        }
        if (k == kEmptyKey) {
            k = atomicCAS(&tab[i].key, kEmptyKey, key);
            if (k == kEmptyKey) {
                atomicAdd(&tab[i].count, c);
                return 1;
            }
            if (k == key) {
                atomicAdd(&tab[i].count, c);
                return 0;
            }
        }
        i = (i + 1u) & mask;
    }
    return -1;
}


// Whole-slot load through L2 (16 bytes: key, count, aux).
__device__ __forceinline__ Slot load_slot(const Slot* s) {
    const ulonglong2 v = __ldcg(reinterpret_cast<const ulonglong2*>(s));
    Slot r;
    r.key = v.x;
    r.count = (unsigned int)v.y;
    r.aux = (unsigned int)(v.y >> 32);
    return r;
}

// Lookup continuing from a loaded first-probe slot `sl` at index i; returns
// the matching slot, or one whose key is kEmptyKey when absent.
__device__ __forceinline__ Slot table_find_from(const Slot* tab, unsigned int mask, unsigned long long key,
                                                unsigned int i, Slot sl, unsigned int max_probe) {
    for (unsigned int p = 0; p < max_probe; ++p) {
        if (sl.key == key || sl.key == kEmptyKey) return sl;
        i = (i + 1u) & mask;
        sl = load_slot(&tab[i]);
    }
    sl.key = kEmptyKey;
    return sl;
}

// Slot index of `key`, or -1 if absent.
__device__ __forceinline__ long long table_find(const Slot* tab, unsigned int mask, unsigned long long key,
                                                unsigned int max_probe) {
    unsigned int i = tile_hash(key) & mask;
    for (unsigned int p = 0; p < max_probe; ++p) {
        const unsigned long long k = tab[i].key;
        if (k == key) return (long long)i;
        if (k == kEmptyKey) return -1;
        i = (i + 1u) & mask;
    }
    return -1;
}

// Union-find over significant-tile indices with parent[v] <= v at all times.
__device__ __forceinline__ int uf_find(int* parent, int v) {
    volatile int* par = parent;
    int p = par[v];
    if (p != v) {
        int prev = v, next;
        while (p > (next = par[p])) {  // strictly decreasing: terminates
            par[prev] = next;          // path halving (benign race)
            prev = p;
            p = next;
        }
    }
    return p;
}

// Root of v without modifying the forest.  Used once all unions are done:
// path halving there could overwrite another thread's freshly written root
// with a stale intermediate ancestor.
__device__ __forceinline__ int uf_root(const int* parent, int v) {
    const volatile int* par = parent;
    int p = par[v];
    while (p != v) {  // parent[v] < v unless v is a root: terminates
        v = p;
        p = par[v];
    }
    return v;
}

// Join the components of a and b; the root with the larger index is hooked
// under the smaller one.  Bounded: returns false if it did not settle.
__device__ __forceinline__ bool uf_unite(int* parent, int a, int b, int limit) {
    int ra = uf_find(parent, a), rb = uf_find(parent, b);
    for (int it = 0; it < limit; ++it) {
        if (ra == rb) return true;
        if (ra < rb) {
            const int ret = atomicCAS(&parent[rb], rb, ra);
            if (ret == rb) return true;
            rb = ret;
        } else {
            const int ret = atomicCAS(&parent[ra], ra, rb);
            if (ret == ra) return true;
            ra = ret;
        }
    }
    return false;
}

// Label code stored in a kept tile's aux after agglomeration: the offset from
// the tile to its cluster-id tile (dx >= 0 because the id tile is the
// (ix, iy)-smallest), or an index into the result's cid array when the offset
// does not fit 15+16 bits.
__device__ __forceinline__ unsigned int label_code(unsigned long long key, unsigned long long cid, unsigned int row) {
    const long long dx = (long long)key_x(key) - (long long)key_x(cid);
    const long long dy = (long long)key_y(key) - (long long)key_y(cid);
    if (dx >= 0 && dx < 32768 && dy >= -32768 && dy < 32768)
        return ((unsigned int)dx << 16) | ((unsigned int)dy & 0xFFFFu);
    return 0x80000000u | row;
}

__device__ __forceinline__ long long label_decode(unsigned long long key, unsigned int code, const long long* cid_rows) {
    if (code == kAuxNone) return (long long)kEmptyKey;  // RASTER_NOISE
    if (code & 0x80000000u) return cid_rows[code & 0x7FFFFFFFu];
    const int dx = (int)(code >> 16);
    const int dy = (int)(short)(code & 0xFFFFu);
    return (long long)pack_key(key_x(key) - dx, key_y(key) - dy);
}

}  // namespace raster
