/*
 * CRAC-FP64 chunk fingerprint -- CPU oracle, plain C.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is part of the oracle that the tests,
 * the smoke check and the benchmark's CPU-baseline leg use to check the CUDA
 * path.  The product library never includes, links or calls it, and it shares
 * no code, header or constant table with the CUDA sources.
 *
 * The paper copies the contents of every active allocation at checkpoint
 * time (Sec. 3.2, "Saving the library-allocated arena") and copies them back
 * at restart.  It has no fingerprint; this project adds one so that a
 * checkpoint can carry only the chunks that changed since the previous one.
 * The function below is a direct transcription of the project's hash
 * definition, one word at a time, with no blocking or reordering:
 *
 *   words:    w_j = little-endian u64 j of the chunk, j = 0..m-1,
 *             m = ceil(len/8), last word zero-padded
 *   per word: x_j = w_j XOR ((j+1)*K1)      (mod 2^64)
 *             y_j = x_j * M1                 (mod 2^64)
 *             f_j = y_j XOR (y_j >> 32)
 *   sum:      acc = sum_j f_j                (mod 2^64)
 *   final:    z = acc XOR (len*M3); z ^= z>>31; z *= M2; z ^= z>>29;
 *             z *= M1; z ^= z>>32;           fp = z
 *
 * Constants (each recomputable with integer square roots):
 *   K1 = floor(2^64 / golden ratio)
 *   M1 = floor(2^64 * frac(sqrt 2)) | 1
 *   M2 = floor(2^64 * frac(sqrt 3)) | 1
 *   M3 = floor(2^64 * frac(sqrt 5)) | 1
 */
#include <stddef.h>
#include <stdint.h>

#define ORACLE_K1 0x9E3779B97F4A7C15ULL
#define ORACLE_M1 0x6A09E667F3BCC909ULL
#define ORACLE_M2 0xBB67AE8584CAA73BULL
#define ORACLE_M3 0x3C6EF372FE94F82BULL

/* Fingerprint of one chunk of len bytes (len >= 1). */
uint64_t oracle_fp64(const uint8_t *p, uint64_t len)
{
    uint64_t m = (len + 7) / 8;
    uint64_t acc = 0;
    for (uint64_t j = 0; j < m; j++) {
        uint64_t w = 0;
        for (uint64_t b = 0; b < 8; b++) {
            uint64_t pos = j * 8 + b;
            if (pos < len)
                w |= (uint64_t)p[pos] << (8 * b);
        }
        uint64_t x = w ^ ((j + 1) * ORACLE_K1);
        uint64_t y = x * ORACLE_M1;
        uint64_t f = y ^ (y >> 32);
        acc += f;
    }
    uint64_t z = acc ^ (len * ORACLE_M3);
    z ^= z >> 31;
    z *= ORACLE_M2;
    z ^= z >> 29;
    z *= ORACLE_M1;
    z ^= z >> 32;
    return z;
}

/* Fingerprints of the ceil(bytes/chunk) chunks of one allocation. */
void oracle_fp_chunks(const uint8_t *p, uint64_t bytes, uint64_t chunk, uint64_t *out)
{
    uint64_t n = (bytes + chunk - 1) / chunk;
    for (uint64_t c = 0; c < n; c++) {
        uint64_t lo = c * chunk;
        uint64_t len = bytes - lo < chunk ? bytes - lo : chunk;
        out[c] = oracle_fp64(p + lo, len);
    }
}
