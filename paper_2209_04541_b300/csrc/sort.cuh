// Radix sorts of the preprocessing passes (device-wide, stable, LSD).
#pragma once

#include <cub/device/device_radix_sort.cuh>

#include "internal.cuh"

namespace pgb {

// Stable sort of (key, value) pairs on key bits [0, end_bit).  The four
// arrays hold `count` entries each; the sorted pairs end up in one array of
// each pair, returned in *keys_out and *vals_out (the other two are free).
template <class K, class V>
void sort_pairs(K* keys, K* keys_alt, V* vals, V* vals_alt, uint64_t count, int end_bit, cudaStream_t s,
                Scratch& scratch, K** keys_out, V** vals_out) {
    cub::DoubleBuffer<K> dk(keys, keys_alt);
    cub::DoubleBuffer<V> dv(vals, vals_alt);
    size_t tmp = 0;
    PGB_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, tmp, dk, dv, (int64_t)count, 0, end_bit, s));
    void* t = scratch.get(tmp, s);
    PGB_CUDA(cub::DeviceRadixSort::SortPairs(t, tmp, dk, dv, (int64_t)count, 0, end_bit, s));
    *keys_out = dk.Current();
    *vals_out = dv.Current();
}

// Lexicographic sort of 32-bit pairs (a[i], b[i]) with a, b < 2^bits: a
// stable sort on b, then a stable sort on a carrying b.  Two rounds of 32-bit
// keys with 32-bit values move as many bytes as one sort of packed 64-bit
// keys over 2 * bits, but each pass of the 32-bit form runs faster (measured
// on 2^28 pairs of 24-bit endpoints: 11.7 ms against 17.0 ms).  On return,
// *a_out and *b_out point at the sorted columns, each one of the four arrays
// (a_alt and b_alt are scratch of the same size).
inline void sort_pairs_lex(uint32_t* a, uint32_t* a_alt, uint32_t* b, uint32_t* b_alt, uint64_t count, int bits,
                           cudaStream_t s, Scratch& scratch, uint32_t** a_out, uint32_t** b_out) {
    uint32_t *k1, *v1;
    sort_pairs(b, b_alt, a, a_alt, count, bits, s, scratch, &k1, &v1);  // by b, carrying a
    uint32_t* k1_free = (k1 == b) ? b_alt : b;
    uint32_t* v1_free = (v1 == a) ? a_alt : a;
    sort_pairs(v1, v1_free, k1, k1_free, count, bits, s, scratch, a_out, b_out);  // by a, carrying b
}

}  // namespace pgb
