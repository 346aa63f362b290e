/*
 * Oracle Philox4x32-10 and the uniform draws built on it -- TEST
 * INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Philox4x32 as published by Salmon, Moraes, Dror and Shaw ("Parallel
 * random numbers: as easy as 1, 2, 3", SC'11): each round multiplies counter
 * words 0 and 2 by two fixed odd 32-bit constants, keeps both halves of the
 * 64-bit products, and permutes/xors them with the other two words and the
 * round key; the key is bumped by the two Weyl constants between rounds.
 *
 * Stream layout (the random draws the paper's Algorithm 1 needs; the paper
 * does not fix a generator): key = (low 32 bits of the seed, high 32 bits of
 * the seed); counter = (coordinate / 4, unit, generation, purpose), lane =
 * coordinate mod 4; u = (r >> 8) * 2^-24, a uniform on [0,1) whose grid makes
 * 2u-1 exact in FP32.
 */
#include "oracle.h"

#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
    uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += PHILOX_W0;
    k1 += PHILOX_W1;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

float orc_uniform(uint64_t seed, uint32_t purpose, uint32_t gen, uint32_t unit, int64_t coord) {
  uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
  uint32_t ctr[4] = {(uint32_t)(coord / 4), unit, gen, purpose};
  uint32_t r[4];
  orc_philox4x32_10(ctr, key, r);
  uint32_t bits = r[coord % 4] >> 8;
  return (float)bits * 0x1p-24f;
}
