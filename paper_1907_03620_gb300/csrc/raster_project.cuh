// Exact projection of a coordinate to its tile index, floor(RN(v * s))
// (Alg. 1 project(); Sect. 3.2), for the CUDA kernels of this library.
#pragma once

namespace raster {

// Projection parameters derived once on the host from the scale s.
struct ProjParams {
    unsigned long long s_odd;  // odd part of the significand of s
    int s_exp;                 // s = s_odd * 2^s_exp
    int s_bits;                // bit length of s_odd
    int d0;                    // 1075 - s_exp: v*s = P * 2^-(d0 - e) for v of biased exponent e
    int top;                   // 52 + s_bits: P = significand(v) * s_odd has top or top+1 bits
    double scale;              // s itself, for the rare FP64 path
    // narrow path (s_bits <= 10): the rounding half-ulp of P for top and for
    // top+1 bits, the bound 2^top between them, and the largest D whose
    // product is still a normal double
    unsigned long long half_lo, half_hi, thr;
    int dmax;
};

// Rare path: the definition itself on the FP64 pipe.
static __device__ __noinline__ bool project_coord_fp64(double v, double scale, int* out) {
    double f = floor(__dmul_rn(v, scale));
    if (!(f >= -2147483647.0 && f <= 2147483646.0)) return false;
    *out = (int)f;
    return true;
}

// floor(RN(v * s)) for one coordinate, exactly.
//
// With P = significand(v) * s_odd (exact) and v*s = P * 2^-D, let F = floor(P * 2^-D)
// and let r be the number of bits of P below its 53 leading ones (the rounding
// position, so ulp = 2^(r-D)).  For a result inside the int32 tile range, ulp < 1,
// F and F+1 are representable, and F+1 has an even significand; hence
//   floor(RN(v*s)) = F + 1  iff  (F + 1) - v*s <= ulp/2    (ties round up to F+1),
//   ceil (RN(v*s)) = F + 1  iff  v*s - F       >  ulp/2    (ties round down to F),
// which is one add of a bias before the shift: (P + bias) >> D.  The first
// gives the tile of a positive coordinate, minus the second that of a negative
// one.  NARROW (s_odd below 2^10, every integer precision 0..4) keeps P below
// 2^63; otherwise the 128-bit product is rounded explicitly.  For a negative
// coordinate NARROW computes F' = (P - half - 1) >> D, so that ceil = F' + 1
// and the tile -(F' + 1) = ~F': both signs take the bias half ^ m and give
// q ^ m with m = 0 or all ones, and share the range bound q <= 2^31 - 2.
template <bool WIDE>
__device__ __forceinline__ bool project_coord(double v, const ProjParams& pp, int* out) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const unsigned int e = (unsigned int)(b >> 52) & 0x7FFu;
    if (e - 1u >= 0x7FEu) {  // zero, subnormal, inf or nan
        if ((b << 1) == 0) {  // +-0 projects to tile 0
            *out = 0;
            return true;
        }
        return project_coord_fp64(v, pp.scale, out);
    }
    const bool neg = (b >> 63) != 0ull;
    const unsigned long long mx = (b & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull;
    unsigned long long q;
    if (!WIDE) {
        const unsigned long long P = mx * (unsigned long long)(unsigned int)pp.s_odd;  // < 2^63 (s_odd < 2^10)
        const int D = pp.d0 - (int)e;                                                 // v*s = P * 2^-D
        if (D <= 0) return false;                                                     // |v*s| >= 2^52
        if (D > pp.dmax) return project_coord_fp64(v, pp.scale, out);  // product below the normal range
        const unsigned long long half = P >= pp.thr ? pp.half_hi : pp.half_lo;
        const unsigned long long m = neg ? ~0ull : 0ull;
        const unsigned long long q = (P + (half ^ m)) >> min(D, 63);  // P + bias < 2^63: a shift of 63 gives 0
        if (q > 2147483646ull) return false;
        *out = (int)((unsigned int)q ^ (unsigned int)m);
        return true;
    } else {
        const unsigned long long lo = mx * pp.s_odd;
        const unsigned long long hi = __umul64hi(mx, pp.s_odd);
        const int t = pp.top + (int)((hi >> (pp.top - 64)) != 0ull);  // 64 <= top <= 105
        const int r = t - 53;                                           // 11..53
        // M = P rounded to 53 significant bits (ties to even), as M * 2^r
        unsigned long long M = (hi << (64 - r)) | (lo >> r);
        const unsigned long long rb = (lo >> (r - 1)) & 1ull;
        const unsigned long long sticky = (lo & ((1ull << (r - 1)) - 1ull)) != 0ull;
        M += rb & (sticky | (M & 1ull));
        const int kk = (int)e - 1075 + pp.s_exp + r;  // RN(v*s) = M * 2^kk
        if (kk < -1074) return project_coord_fp64(v, pp.scale, out);
        const int D = -kk;
        if (D <= 0) return false;
        if (D >= 64) {
            q = neg ? 1ull : 0ull;
        } else {
            const unsigned long long ip = M >> D;
            const unsigned long long fr = (M << (64 - D)) != 0ull;
            q = neg ? ip + fr : ip;
        }
    }
    if (neg) {
        if (q > 2147483647ull) return false;
        *out = -(int)q;
    } else {
        if (q > 2147483646ull) return false;
        *out = (int)q;
    }
    return true;
}

}  // namespace raster
