// catfhe_rescale_noalloc: the CKKS rescale / BGV modulus switch for callers
// that may not allocate device memory.
//
// Some callers cannot call cudaMalloc while they work: code that runs inside
// a host callback or a signal-safe section, a serving loop with a fixed
// memory budget fixed at start-up, or a plugin whose host process owns every
// device allocation.  catfhe_rescale needs a workspace (either passed in or
// grown by the context), so such a caller has nowhere to put it.  This entry
// point takes its scratch from kNoallocBytes of device memory that the
// library reserves statically (a file-scope __device__ array): every GPU
// that loads the library holds that memory until the process exits, and no
// call here allocates or frees anything.
//
// The array has no device address in host code (its name there is only a
// host-side stand-in), so the first call on each device looks the address
// up with cudaGetSymbolAddress while that device is current and keeps it.
// All calls share the one array and it keeps the last call's contents;
// calls whose device work overlaps (two streams, or two host threads) race
// on it and must be ordered by the caller.
#include <mutex>

#include "modarith.cuh"

namespace catfhe {

int op_rescale_noalloc_impl(Context &c, const uint64_t *a, uint64_t *out, uint32_t level,
                            uint32_t count, cudaStream_t s);

// 32 MiB: room for one N = 2^16 ciphertext at 24 primes (plus the plan).
constexpr size_t kNoallocBytes = size_t(32) << 20;
constexpr size_t kNoallocPlanBytes = 16 << 10;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

static std::mutex g_noalloc_mu;
static void *g_noalloc_ptr[64];  // device address of the array, per device

// Device address of the static scratch on the context's device (looked up
// once per device).  The array's address differs per device, so the caller's
// current device must be the context's: otherwise the kernels would get
// another GPU's array with no error, and the call is refused instead.
static int noalloc_scratch(const Context &c, void **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return CATFHE_ECUDA;
    if (dev != c.device) return CATFHE_EINVAL;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return CATFHE_ECUDA;
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return CATFHE_OK;
}

// Layout of the scratch for count ciphertexts at `level`: the plan, then the
// inverse-transformed last limbs [count][2][N], then the lift
// [count][2][level-1][N].  The size check and the call use these same
// offsets, so the check covers every word the kernels touch:
// 16 KiB + 16 count level N bytes in all.
struct NoallocLayout {
    size_t last_off, lift_off, end;
};

static NoallocLayout noalloc_layout(const Context &c, uint32_t level, uint32_t count) {
    NoallocLayout l;
    const size_t lo = level >= 1 ? level - 1 : 0;
    l.last_off = kNoallocPlanBytes;
    l.lift_off = l.last_off + size_t(count) * 2 * c.n * 8;
    l.end = l.lift_off + size_t(count) * 2 * lo * c.n * 8;
    return l;
}

// The rescale plan (one source prime q_{l-1}, targets q_0 .. q_{l-2}) in the
// Montgomery layout, written into a fixed host buffer.
static size_t rescale_plan(const Context &c, uint32_t lvl, uint64_t *buf) {
    const uint32_t T = lvl - 1;
    const uint64_t m = c.mod(int(lvl) - 1);
    const bool bgv = c.scheme == CATFHE_BGV;
    const uint64_t pre = bgv ? h_invmod(c.t % m, m) : 1;
    auto neg_inv = [](uint64_t x) {
        uint64_t y = x;
        for (int i = 0; i < 6; i++) y *= 2 - x * y;
        return 0 - y;
    };
    auto r64 = [](uint64_t x) { return (uint64_t)(((unsigned __int128)1 << 64) % x); };
    size_t w = 0;
    buf[w++] = uint64_t(1) | (uint64_t(T) << 16) | (uint64_t(1) << 33) | (uint64_t(1) << 34);
    buf[w++] = 0;                                         // src_off
    for (uint32_t t = 0; t < T; t++) buf[w++] = t;        // dst_off
    buf[w++] = m;                                         // smod
    buf[w++] = neg_inv(m);
    for (uint32_t t = 0; t < T; t++) {                    // dmod
        buf[w++] = c.mod(int(t));
        buf[w++] = neg_inv(c.mod(int(t)));
    }
    buf[w++] = h_mulmod(pre, r64(m), m);                  // C[0][0]
    buf[w++] = (m - 1) / 2;                               // h[0]
    for (uint32_t t = 0; t < T; t++) {                    // Ct[0][t]
        const uint64_t p = c.mod(int(t));
        const uint64_t post = bgv ? c.t % p : 1;
        buf[w++] = h_mulmod(post, r64(p), p);
    }
    for (uint32_t t = 0; t < T; t++) {                    // Mneg[t]
        const uint64_t p = c.mod(int(t));
        const uint64_t post = bgv ? c.t % p : 1;
        buf[w++] = h_mulmod(h_mulmod((p - m % p) % p, post, p), r64(p), p);
    }
    return w;
}

int op_rescale_noalloc_impl(Context &c, const uint64_t *a, uint64_t *out, uint32_t level,
                            uint32_t count, cudaStream_t s) {
    if (c.scheme == CATFHE_BFV) return CATFHE_ESCHEME;
    if (level < 2 || int(level) > c.L) return CATFHE_ELEVEL;
    if (count == 0) return CATFHE_OK;
    const NoallocLayout lay = noalloc_layout(c, level, count);
    if (lay.end > kNoallocBytes) return CATFHE_EWORKSPACE;
    // the combine reads a with a stride of 2 level N words and writes out with
    // 2 (level-1) N: overlapping spans would overwrite inputs before they are read
    const uintptr_t a0 = reinterpret_cast<uintptr_t>(a), o0 = reinterpret_cast<uintptr_t>(out);
    const size_t a_bytes = size_t(count) * 2 * level * c.n * 8;
    const size_t o_bytes = size_t(count) * 2 * (level - 1) * c.n * 8;
    if (a0 < o0 + o_bytes && o0 < a0 + a_bytes) return CATFHE_EINVAL;
    void *base = nullptr;
    int rc = noalloc_scratch(c, &base);
    if (rc) return rc;
    const size_t n = c.n;
    const int lvl = int(level), lo = lvl - 1;
    char *b8 = static_cast<char *>(base);
    uint64_t *plan = reinterpret_cast<uint64_t *>(b8);
    uint64_t *last = reinterpret_cast<uint64_t *>(b8 + lay.last_off);
    uint64_t *lift = reinterpret_cast<uint64_t *>(b8 + lay.lift_off);

    uint64_t hplan[1 + 1 + 32 + 2 + 64 + 2 + 32 + 32];
    const size_t words = rescale_plan(c, level, hplan);
    if (cudaMemcpyAsync(plan, hplan, words * 8, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return CATFHE_ECUDA;
    // INTT of the last limb of both polynomials into the scratch
    LimbMap m{};
    m.period = 2;
    m.src_stride = uint32_t(2 * lvl);
    m.dst_stride = 2;
    for (int p = 0; p < 2; p++) {
        m.src_off[p] = uint16_t(p * lvl + lvl - 1);
        m.dst_off[p] = uint16_t(p);
        m.prime[p] = uint8_t(lvl - 1);
    }
    if ((rc = launch_ntt_inv(c, a, last, m, 2 * count, s))) return rc;
    PlanList pl{};
    pl.n = 1;
    pl.kmax = 1;
    pl.kmin = 1;
    pl.words = uint32_t(words);
    pl.mont = 1;
    pl.p[0] = plan;
    if ((rc = launch_conv(c, pl, last, n, 0, lift, size_t(lo) * n, 0, 2 * count, s))) return rc;
    LimbMap ml{};
    ml.period = uint32_t(lo);
    ml.src_stride = ml.dst_stride = uint32_t(lo);
    for (int i = 0; i < lo; i++) {
        ml.src_off[i] = ml.dst_off[i] = uint16_t(i);
        ml.prime[i] = uint8_t(i);
    }
    if ((rc = launch_ntt_fwd(c, lift, lift, ml, uint32_t(2 * lo) * count, s))) return rc;
    CombineArgs ca{};
    ca.y = a;
    ca.lift = lift;
    ca.out = out;
    ca.y_item = size_t(2) * lvl * n;
    ca.y_poly = size_t(lvl) * n;
    ca.lift_item = size_t(2) * lo * n;
    ca.lift_poly = size_t(lo) * n;
    ca.out_item = size_t(2) * lo * n;
    ca.out_poly = size_t(lo) * n;
    ca.lo = uint32_t(lo);
    for (int i = 0; i < lo; i++) {
        ca.prime[i] = uint8_t(i);
        ca.dinv[i] = h_invmod(c.mod(lvl - 1) % c.mod(i), c.mod(i));
        ca.dinv_s[i] = h_shoup(ca.dinv[i], c.mod(i));
    }
    return launch_combine(c, ca, count, s);
}

}  // namespace catfhe
