/*
 * The counter-based random stream and relabelling bijection of the seeded
 * graph generators, shared by the host generators (graphgen.c, gcc) and the
 * device generators (graphgen_dev.cu, nvcc) so that both write the same
 * graphs edge for edge.  Input plumbing only: nothing here belongs to the
 * triangle-counting method.
 *
 * Stream: SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom
 * number generators", OOPSLA 2014).  Draw c of the stream keyed by `key` is
 *     mix(key + (c + 1) * 0x9E3779B97F4A7C15),
 * mix() being SplitMix64's output function; a generator's key is
 * mix(seed ^ tag) for a per-generator tag.
 *
 * Relabelling: a 4-round Feistel network on the `bits`-bit vertex IDs (Luby
 * and Rackoff's construction).  The ID splits into a high half of
 * floor(bits / 2) bits and a low half of the rest; round r (0..3) XORs into
 * one half (the high half in even rounds, the low half in odd ones) the high
 * 32 bits of draw (r << 32 | other half) of the stream keyed by
 * mix(seed ^ "FEIS"), masked to the half's width.  Each round is its own
 * inverse, so the whole map is a bijection on [0, 2^bits) that every thread
 * evaluates on its own.
 */
#ifndef GG_STREAM_H
#define GG_STREAM_H

#include <stdint.h>

#ifdef __CUDACC__
#define GG_HD __host__ __device__ __forceinline__
#else
#define GG_HD static inline
#endif

#define GG_GOLDEN 0x9E3779B97F4A7C15ULL
#define GG_TAG_FEISTEL 0x46454953ULL

GG_HD uint64_t gg_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Draw number c of the stream keyed by key. */
GG_HD uint64_t gg_draw(uint64_t key, uint64_t c) { return gg_mix(key + (c + 1) * GG_GOLDEN); }

/* Uniform integer in [0, n) from 32 random bits (Lemire's multiply-shift;
 * bias below n / 2^32). */
GG_HD uint32_t gg_below(uint32_t x32, uint32_t n) { return (uint32_t)(((uint64_t)x32 * (uint64_t)n) >> 32); }

/* The Feistel relabelling of x in [0, 2^bits), 1 <= bits <= 31, under the
 * stream key fkey = mix(seed ^ GG_TAG_FEISTEL). */
GG_HD uint32_t gg_feistel(uint32_t x, uint32_t bits, uint64_t fkey) {
    const uint32_t hb = bits / 2, lb = bits - hb;
    const uint32_t hmask = hb ? (uint32_t)((1ull << hb) - 1) : 0u, lmask = (uint32_t)((1ull << lb) - 1);
    uint32_t hi = (x >> lb) & hmask, lo = x & lmask;
    for (uint32_t r = 0; r < 4; ++r) {
        if ((r & 1u) == 0) hi ^= (uint32_t)(gg_draw(fkey, ((uint64_t)r << 32) | lo) >> 32) & hmask;
        else lo ^= (uint32_t)(gg_draw(fkey, ((uint64_t)r << 32) | hi) >> 32) & lmask;
    }
    return (hi << lb) | lo;
}

/* R-MAT quadrant thresholds for 32-bit uniforms: r < ta top-left, r < tb
 * top-right, r < tc bottom-left, else bottom-right. */
GG_HD void gg_rmat_thresholds(double a, double b, double c, uint64_t* ta, uint64_t* tb, uint64_t* tc) {
    *ta = (uint64_t)(a * 4294967296.0);
    *tb = (uint64_t)((a + b) * 4294967296.0);
    *tc = (uint64_t)((a + b + c) * 4294967296.0);
}

/* Edge e of an R-MAT graph on 2^scale vertices (before relabelling): level
 * lvl (most significant bit first) takes one 32-bit uniform, the high half
 * of draw e * ceil(scale / 2) + lvl / 2 at even levels and its low half at
 * odd ones. */
GG_HD void gg_rmat_edge(uint64_t key, uint32_t scale, uint64_t e, uint64_t ta, uint64_t tb, uint64_t tc,
                        uint32_t* src, uint32_t* dst) {
    const uint64_t draws_per_edge = (scale + 1) / 2;
    uint32_t s = 0, d = 0;
    uint64_t x = 0;
    for (uint32_t lvl = 0; lvl < scale; ++lvl) {
        uint32_t r;
        if ((lvl & 1u) == 0) {
            x = gg_draw(key, e * draws_per_edge + lvl / 2);
            r = (uint32_t)(x >> 32);
        } else {
            r = (uint32_t)x;
        }
        const uint32_t bit = 1u << (scale - 1 - lvl);
        if (r < ta) {
        } else if (r < tb) {
            d |= bit;
        } else if (r < tc) {
            s |= bit;
        } else {
            s |= bit;
            d |= bit;
        }
    }
    *src = s;
    *dst = d;
}

#endif
