/* Fast fills for the seeded input generator (paper_1511_06441_gb300/synth.py).
 *
 * Counter-based SplitMix64 (Steele, Lea & Flood 2014): value i of stream s under seed k
 * is mix(base + (i + 1) * GAMMA) with base = mix(k * 0x2545F4914F6CDD1D + s).  Same
 * definition as synth.u64; the tests check that both give identical arrays.  Random
 * numbers only: nothing of the solver's arithmetic is here.
 */
#include <stdint.h>

static uint64_t mix(uint64_t z)
{
    z ^= z >> 30;
    z *= 0xBF58476D1CE4E5B9ull;
    z ^= z >> 27;
    z *= 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* out[i] = lo + u64(seed, stream, i + offset) mod (hi - lo + 1), i < n, as 1, 2 or 8 bytes;
 * entries whose mask byte is nonzero are set to 0 instead (mask nullable). */
void synth_fill_uniform(uint64_t seed, uint64_t stream, int64_t n, int64_t offset, int64_t lo, int64_t hi,
                        const uint8_t *mask, void *out, int out_bytes)
{
    const uint64_t base = mix(seed * 0x2545F4914F6CDD1Dull + stream);
    const uint64_t span = (uint64_t)(hi - lo + 1);
    for (int64_t i = 0; i < n; i++) {
        uint64_t x = mix(base + (uint64_t)(i + offset + 1) * 0x9E3779B97F4A7C15ull);
        int64_t v = lo + (int64_t)(x % span);
        if (mask && mask[i]) v = 0;
        if (out_bytes == 1) ((uint8_t *)out)[i] = (uint8_t)v;
        else if (out_bytes == 2) ((uint16_t *)out)[i] = (uint16_t)v;
        else ((int64_t *)out)[i] = v;
    }
}

/* mask[k*V + v] = 1 where coordinate k of v is extents[k] - 1 (the edge leaves the box). */
void synth_upper_face_mask(int d, const int64_t *extents, uint8_t *mask)
{
    int64_t V = 1;
    for (int k = 0; k < d; k++) V *= extents[k];
    int64_t stride = 1;
    for (int k = 0; k < d; k++) {
        for (int64_t v = 0; v < V; v++) mask[k * V + v] = ((v / stride) % extents[k]) == extents[k] - 1;
        stride *= extents[k];
    }
}
