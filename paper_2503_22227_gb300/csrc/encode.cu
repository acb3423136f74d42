// CKKS encoding and decoding on the device (Table 1 "encode" / "decode"):
// the canonical embedding evaluates the plaintext polynomial m at the
// primitive 2N-th roots zeta^(5^k) (slot k < N/2) and their conjugates.
// With zeta = exp(i pi / N) and omega = zeta^2,
//     m(zeta^(2j+1)) = sum_i (m_i zeta^i) omega^(i j),
// so all N evaluations are one length-N DFT of the twisted coefficients:
//   encode: E[j(k)] = scale z_k, E[j'(k)] = conj(scale z_k) (j = (5^k - 1)/2,
//           j' = (2N - 5^k - 1)/2), then m_i = round(Re(zeta^-i IDFT(E)_i));
//   decode: z_k = DFT(m_i zeta^i)[j(k)] / scale.
// This is the only floating-point stage of the library (float64); the
// result is rounded to integers before any modular arithmetic.  The DFT is
// an iterative radix-2 transform (bit-reversal copy, then log2 N butterfly
// passes of N/2 threads): the vectors are small (N complex doubles) and the
// transform runs once per encoded or decoded message.
#include <math.h>

#include <vector>

#include "modarith.cuh"

namespace catfhe {

namespace {

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__global__ void k_scatter_slots(const double2 *__restrict__ z, double scale,
                                const uint32_t *__restrict__ idx, double2 *E, uint32_t half) {
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= half) return;
    const double2 v = make_double2(scale * z[k].x, scale * z[k].y);
    E[idx[k]] = v;
    E[idx[half + k]] = make_double2(v.x, -v.y);
}

__global__ void k_bitrev(const double2 *__restrict__ in, double2 *__restrict__ out,
                         uint32_t log_n) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >> log_n) return;
    out[__brev(i) >> (32 - log_n)] = in[i];
}

// One radix-2 pass: butterflies of span `half` with twiddles tw[pos * N / (2 half)].
__global__ void k_fft_pass(double2 *x, const double2 *__restrict__ tw, uint32_t lg_half,
                           uint32_t log_n) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >> (log_n - 1)) return;
    const uint32_t half = 1u << lg_half;
    const uint32_t pos = t & (half - 1), grp = t >> lg_half;
    const uint32_t i0 = (grp << (lg_half + 1)) + pos, i1 = i0 + half;
    const double2 w = tw[pos << (log_n - 1 - lg_half)];
    const double2 a = x[i0], b = cmul(w, x[i1]);
    x[i0] = make_double2(a.x + b.x, a.y + b.y);
    x[i1] = make_double2(a.x - b.x, a.y - b.y);
}

__global__ void k_untwist_round(const double2 *__restrict__ x, const double2 *__restrict__ twist,
                                double inv_n, int64_t *m, uint32_t n) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    // Re(x_i conj(zeta^i)) / N, rounded half away from zero
    const double v = (x[i].x * twist[i].x + x[i].y * twist[i].y) * inv_n;
    m[i] = (int64_t)round(v);
}

__global__ void k_twist(const int64_t *__restrict__ m, const double2 *__restrict__ twist, double2 *x,
                        uint32_t n) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double v = double(m[i]);
    x[i] = make_double2(v * twist[i].x, v * twist[i].y);
}

__global__ void k_gather_slots(const double2 *__restrict__ X, const uint32_t *__restrict__ idx,
                               double inv_scale, double2 *z, uint32_t half) {
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= half) return;
    const double2 v = X[idx[k]];
    z[k] = make_double2(v.x * inv_scale, v.y * inv_scale);
}

inline unsigned blocks(size_t n) { return unsigned((n + 255) / 256); }

// x (N complex) <- DFT with twiddles tw (omega^(+-k), k < N/2), via tmp.
int dft(const Context &c, const double2 *in, double2 *out, const double2 *tw, cudaStream_t s) {
    const uint32_t lg = uint32_t(c.log_n);
    k_bitrev<<<blocks(c.n), 256, 0, s>>>(in, out, lg);
    for (uint32_t h = 0; h < lg; h++) k_fft_pass<<<blocks(c.n / 2), 256, 0, s>>>(out, tw, h, lg);
    note_launches(1 + lg);
    return cudaGetLastError() == cudaSuccess ? CATFHE_OK : CATFHE_ECUDA;
}

}  // namespace

// Tables: d_enc = [twist zeta^i (N)][omega^k (N/2)][omega^-k (N/2)],
// d_slot = [j(k) (N/2)][j'(k) (N/2)].
int enc_tables(Context &c) {
    if (c.d_enc) return CATFHE_OK;
    const size_t n = c.n, half = n / 2;
    std::vector<double2> h(2 * n);
    const double pi = 3.14159265358979323846;
    for (size_t i = 0; i < n; i++) h[i] = make_double2(cos(pi * double(i) / double(n)), sin(pi * double(i) / double(n)));
    for (size_t k = 0; k < half; k++) {
        const double a = 2 * pi * double(k) / double(n);
        h[n + k] = make_double2(cos(a), sin(a));
        h[n + half + k] = make_double2(cos(a), -sin(a));
    }
    std::vector<uint32_t> idx(n);
    uint64_t e = 1;
    for (size_t k = 0; k < half; k++) {
        idx[k] = uint32_t((e - 1) / 2);
        idx[half + k] = uint32_t((2 * n - e - 1) / 2);
        e = e * 5 % (2 * n);
    }
    double2 *d = nullptr;
    uint32_t *di = nullptr;
    if (cudaMalloc(&d, h.size() * sizeof(double2)) != cudaSuccess) return CATFHE_ENOMEM;
    if (cudaMalloc(&di, idx.size() * 4) != cudaSuccess) {
        cudaFree(d);
        return CATFHE_ENOMEM;
    }
    if (cudaMemcpy(d, h.data(), h.size() * sizeof(double2), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(di, idx.data(), idx.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(d);
        cudaFree(di);
        return CATFHE_ECUDA;
    }
    c.d_enc = d;
    c.d_slot = di;
    return CATFHE_OK;
}

int launch_encode_ckks(const Context &c, const double2 *slots, double scale, double2 *buf0,
                       double2 *buf1, int64_t *m, cudaStream_t s) {
    const size_t n = c.n, half = n / 2;
    const double2 *twist = c.d_enc, *tw_inv = c.d_enc + n + half;
    k_scatter_slots<<<blocks(half), 256, 0, s>>>(slots, scale, c.d_slot, buf0, uint32_t(half));
    note_launches(1);
    const int rc = dft(c, buf0, buf1, tw_inv, s);
    if (rc) return rc;
    k_untwist_round<<<blocks(n), 256, 0, s>>>(buf1, twist, 1.0 / double(n), m, uint32_t(n));
    note_launches(1);
    return cudaGetLastError() == cudaSuccess ? CATFHE_OK : CATFHE_ECUDA;
}

int launch_decode_ckks(const Context &c, const int64_t *m, double inv_scale, double2 *buf0,
                       double2 *buf1, double2 *slots, cudaStream_t s) {
    const size_t n = c.n, half = n / 2;
    const double2 *twist = c.d_enc, *tw_fwd = c.d_enc + n;
    k_twist<<<blocks(n), 256, 0, s>>>(m, twist, buf0, uint32_t(n));
    note_launches(1);
    const int rc = dft(c, buf0, buf1, tw_fwd, s);
    if (rc) return rc;
    k_gather_slots<<<blocks(half), 256, 0, s>>>(buf1, c.d_slot, inv_scale, slots, uint32_t(half));
    note_launches(1);
    return cudaGetLastError() == cudaSuccess ? CATFHE_OK : CATFHE_ECUDA;
}

}  // namespace catfhe
