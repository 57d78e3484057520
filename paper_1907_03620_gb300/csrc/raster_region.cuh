// Region-partitioned tile table for the single-instance path.
//
// The table is split into `regions` regions of 2^region_bits slots.  A tile's
// home slot is in the region chosen by a hash of its 16 x 16-tile spatial
// block, at an offset chosen by a hash of the tile itself.  Each region is a
// whole number of buckets of 2^kBucketBits slots (64 KiB), and probing is
// linear within the home bucket, wrapping at its end.  Two consequences shape
// the kernels:
//   * the eight neighbours of a tile almost always share its region, so the
//     agglomeration's neighbour probes (which walk significant tiles in slot
//     order) and its union-find accesses stay within a few regions at a time
//     and hit L2;
//   * contraction sorts a round's keys by region and then by bucket, and
//     inserts each bucket's keys into a copy of the bucket in shared memory,
//     so the table is read and written once per round, in whole buckets.
#pragma once

#include "raster_device.cuh"

namespace raster {

constexpr int kBlockShift = 4;  // spatial blocks of 16 x 16 tiles
constexpr int kBucketBits = 12;  // probing stays within 4096-slot buckets
constexpr unsigned int kBucketSlots = 1u << kBucketBits;

struct RegionTable {
    Slot* tab;
    unsigned long long cap;  // regions << region_bits
    unsigned int regions;
    unsigned int region_bits;
    unsigned int max_probe;
    int dims;  // coordinates of the keys: 2, or 3 (spatial blocks of 8 x 8 x 8 tiles)
};

__device__ __forceinline__ unsigned int block_hash(unsigned long long key) {
    const unsigned int bx = (unsigned int)(key_x(key) >> kBlockShift);  // floor division for negative indices
    const unsigned int by = (unsigned int)(key_y(key) >> kBlockShift);
    unsigned int h = bx * 0x9E3779B1u + by * 0x85EBCA77u;
    h ^= h >> 15;
    h *= 0x2C1B3C6Du;
    h ^= h >> 12;
    h *= 0x297A2D39u;
    h ^= h >> 15;
    return h;
}

__device__ __forceinline__ unsigned int block_hash3(unsigned long long key) {
    const unsigned int bx = (unsigned int)(key3(key, 0) >> 3), by = (unsigned int)(key3(key, 1) >> 3);
    const unsigned int bz = (unsigned int)(key3(key, 2) >> 3);
    unsigned int h = bx * 0x9E3779B1u + by * 0x85EBCA77u + bz * 0xC2B2AE3Du;
    h ^= h >> 15;
    h *= 0x2C1B3C6Du;
    h ^= h >> 12;
    h *= 0x297A2D39u;
    h ^= h >> 15;
    return h;
}

__device__ __forceinline__ unsigned int region_of(unsigned long long key, const RegionTable& t) {
    const unsigned int h = t.dims == 3 ? block_hash3(key) : block_hash(key);
    return (unsigned int)(((unsigned long long)h * t.regions) >> 32);
}

__device__ __forceinline__ unsigned long long home_slot(unsigned long long key, const RegionTable& t) {
    return ((unsigned long long)region_of(key, t) << t.region_bits) |
           (unsigned long long)(tile_hash(key) & ((1u << t.region_bits) - 1u));
}

__device__ __forceinline__ unsigned long long next_slot(unsigned long long i, const RegionTable&) {
    return (i & ~(unsigned long long)(kBucketSlots - 1u)) | ((i + 1ull) & (kBucketSlots - 1u));
}

// Add c points to `key`: 1 if new, 0 if present, -1 if max_probe slots failed.
__device__ __forceinline__ int rt_add(const RegionTable& t, unsigned long long key, unsigned int c) {
    unsigned long long i = home_slot(key, t);
    for (unsigned int p = 0; p < t.max_probe; ++p) {
        unsigned long long k = load_key(&t.tab[i]);
        if (k == key) {
            atomicAdd(&t.tab[i].count, c);
            return 0;
        }
        if (k == kEmptyKey) {
            k = atomicCAS(&t.tab[i].key, kEmptyKey, key);
            if (k == kEmptyKey || k == key) {
                atomicAdd(&t.tab[i].count, c);
                return k == kEmptyKey ? 1 : 0;
            }
        }
        i = next_slot(i, t);
    }
    return -1;
}

// The slot holding `key` (whole 16 bytes), or one with key kEmptyKey if absent.
__device__ __forceinline__ Slot rt_lookup(const RegionTable& t, unsigned long long key, unsigned long long i, Slot sl) {
    for (unsigned int p = 0; p < t.max_probe; ++p) {
        if (sl.key == key || sl.key == kEmptyKey) return sl;
        i = next_slot(i, t);
        sl = load_slot(&t.tab[i]);
    }
    sl.key = kEmptyKey;
    return sl;
}

__device__ __forceinline__ Slot rt_get(const RegionTable& t, unsigned long long key) {
    const unsigned long long i = home_slot(key, t);
    return rt_lookup(t, key, i, load_slot(&t.tab[i]));
}

// The slot index of `key`, or -1 when it is absent.
__device__ __forceinline__ long long rt_find(const RegionTable& t, unsigned long long key) {
    unsigned long long i = home_slot(key, t);
    for (unsigned int p = 0; p < t.max_probe; ++p) {
        const unsigned long long k = t.tab[i].key;
        if (k == key) return (long long)i;
        if (k == kEmptyKey) return -1;
        i = next_slot(i, t);
    }
    return -1;
}

}  // namespace raster
