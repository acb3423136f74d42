// Bit-packed transfer form of ciphertexts (host <-> device), an addition of
// this library (the paper moves ciphertexts in whole words).  Each limb's N
// residues of prime q_i travel as a little-endian bit stream of
// b_i = bitlen(q_i) bits per residue: residue k occupies bits
// [k b_i, (k+1) b_i) of the limb's N b_i / 64 words.  Limbs keep the at-rest
// order [count][2][level] and the at-rest form (NTT form for CKKS and BGV).
// A residue below q_i < 2^b_i leaves 64 - b_i bits of every at-rest word
// empty; for the 50-bit primes of the N = 2^16 chain the packed form is 22%
// smaller, and the host link is the bound of an end-to-end step.
#include "internal.h"
#include "launch.cuh"
#include "modarith.cuh"

namespace catfhe {

// bits[i], q[i] and the word offset off[i] of limb i inside one
// polynomial's packed block (off[level] = the block's size).
struct PackArgs {
    uint32_t level, log_n;
    uint32_t bits[kConvMaxK];
    uint64_t q[kConvMaxK];
    uint64_t off[kConvMaxK + 1];
};

// One residue per thread; reads the one or two words holding its bits.  A
// value of b_i bits is below 2 q_i (q_i >= 2^(b_i - 1)): one conditional
// subtraction makes any packed input a valid residue (valid inputs pass
// unchanged).
__global__ void __launch_bounds__(256) k_unpack(const uint64_t *__restrict__ packed,
                                                uint64_t *__restrict__ out, const PackArgs A) {
    grid_dep_wait();
    const uint32_t i = blockIdx.y, poly = blockIdx.z;
    const size_t n = size_t(1) << A.log_n;
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const uint32_t b = A.bits[i];
    const uint64_t *src = packed + size_t(poly) * A.off[A.level] + A.off[i];
    const uint64_t o = uint64_t(k) * b;
    const uint32_t w = uint32_t(o >> 6), sh = uint32_t(o & 63);
    uint64_t v = src[w] >> sh;
    if (sh + b > 64) v |= src[w + 1] << (64 - sh);
    if (b < 64) v &= (uint64_t(1) << b) - 1;
    out[(size_t(poly) * A.level + i) * n + k] = csub(v, A.q[i]);
}

// One packed word per thread: the residues whose bits meet word w.
__global__ void __launch_bounds__(256) k_pack(const uint64_t *__restrict__ in,
                                              uint64_t *__restrict__ packed, const PackArgs A) {
    grid_dep_wait();
    const uint32_t i = blockIdx.y, poly = blockIdx.z;
    const size_t n = size_t(1) << A.log_n;
    const uint32_t b = A.bits[i];
    const uint32_t words = uint32_t(A.off[i + 1] - A.off[i]);
    const uint32_t w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= words) return;
    const uint64_t *src = in + (size_t(poly) * A.level + i) * n;
    const uint64_t lo = uint64_t(w) * 64;
    const uint32_t k0 = uint32_t(lo / b);
    const uint64_t k_last = (lo + 63) / b;
    const uint32_t k1 = uint32_t(k_last < n - 1 ? k_last : n - 1);
    uint64_t word = 0;
    for (uint32_t k = k0; k <= k1; k++) {
        const int64_t pos = int64_t(uint64_t(k) * b) - int64_t(lo);  // in (-b, 64)
        const uint64_t v = src[k];
        word |= pos >= 0 ? v << pos : v >> (-pos);
    }
    packed[size_t(poly) * A.off[A.level] + A.off[i] + w] = word;
}

static PackArgs pack_args(const Context &c, uint32_t level) {
    PackArgs a{};
    a.level = level;
    a.log_n = uint32_t(c.log_n);
    uint64_t off = 0;
    for (uint32_t i = 0; i < level; i++) {
        const uint64_t q = c.mod(int(i));
        uint32_t b = 0;
        while (b < 64 && (q >> b) != 0) b++;
        a.bits[i] = b;
        a.q[i] = q;
        a.off[i] = off;
        off += (c.n * b) / 64;
    }
    a.off[level] = off;
    return a;
}

size_t packed_words(const Context &c, uint32_t level) { return pack_args(c, level).off[level]; }

int launch_unpack(const Context &c, const uint64_t *packed, uint64_t *out, uint32_t level,
                  uint32_t polys, cudaStream_t s) {
    const PackArgs a = pack_args(c, level);
    launch_pdl(k_unpack, dim3(unsigned((c.n + 255) / 256), level, polys), dim3(256), 0, s, packed,
               out, a);
    note_launches(1);
    return cudaGetLastError() == cudaSuccess ? CATFHE_OK : CATFHE_ECUDA;
}

int launch_pack(const Context &c, const uint64_t *in, uint64_t *packed, uint32_t level,
                uint32_t polys, cudaStream_t s) {
    const PackArgs a = pack_args(c, level);
    launch_pdl(k_pack, dim3(unsigned((c.n + 255) / 256), level, polys), dim3(256), 0, s, in,
               packed, a);
    note_launches(1);
    return cudaGetLastError() == cudaSuccess ? CATFHE_OK : CATFHE_ECUDA;
}

}  // namespace catfhe
