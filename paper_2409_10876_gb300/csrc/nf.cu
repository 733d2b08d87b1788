// Neural-field SOS on fifth-generation tensor cores (sm_103a tcgen05, BF16
// operands, FP32 accumulation in tensor memory).
//
// The field (the coordinate-based SOS representation of Sec. 3.3, here the
// Fourier-feature MLP of the BF16 workload) maps every SOS node to
//   f(x, y) = [sin 2pi f_l x, cos 2pi f_l x, sin 2pi f_l y, cos 2pi f_l y]_l  (64)
//   h1..h4 = relu(W h + b)  (128 each),   z = w5 . h4 + b5,
//   v = v_mid + v_half tanh z  inside the mask, v_bg outside,
// with x, y the node position over the field of view and f_l = 64^(l/15).
//
// pact_nf_forward: one CTA per 128 nodes; the four hidden layers are four
// 128 x 128 (x 64 / 128) GEMMs on the tensor cores with the accumulator in
// TMEM; each thread owns one node (one TMEM lane) for the bias/ReLU epilogue,
// which writes the next layer's operand straight into shared memory.  The BF16
// weights are cast into their operand-tile layout once per call, so each tile
// arrives by one bulk copy (TMA) on its own mbarrier; each layer's output tile
// goes (in its shared-memory layout) to the workspace for the backward pass by
// one bulk store that runs while the next layer computes.
// pact_nf_backward: per CTA and layer, dW = dz^T h (M = out, N = in, K = 128
// nodes; dz and h are the K-major node tiles read as MN-major operands, so no
// transposed copies) and dh = dz W (M = nodes, N = in, K = out) on the tensor
// cores, the layer's h and W tiles arriving by bulk copies into a second buffer
// pair while the layer before runs; the per-CTA weight gradients go to the
// workspace (coalesced, [in/4][out][4] per block) and a second kernel sums
// them in a fixed order.
#include <math.h>

#include <algorithm>

#include "pact_internal.cuh"
#include "umma.cuh"

namespace pact {
namespace {

constexpr int kF = 64;      // Fourier features
constexpr int kH = 128;     // hidden width
constexpr int kL = 4;       // hidden layers
constexpr int kRows = 128;  // nodes per CTA (one TMEM lane each)

__host__ __device__ constexpr int in_dim(int l) { return l == 1 ? kF : kH; }
__host__ __device__ constexpr int off_w(int l) { return l == 1 ? 0 : kH * kF + kH + (l - 2) * (kH * kH + kH); }
__host__ __device__ constexpr int off_b(int l) { return off_w(l) + kH * in_dim(l); }
constexpr int kOffW5 = off_w(kL + 1);
constexpr int kOffB5 = kOffW5 + kH;
constexpr int kNParam = kOffB5 + 1;
constexpr int kPartStride = (kNParam + 63) / 64 * 64;   // per-CTA gradient row, 256-byte aligned
constexpr int kTileBytes = kRows * kH * 2;    // one 128 x 128 bf16 operand tile
constexpr int kOnesBytes = 16 * kRows * 2;    // the backward's [16 x 128] tile of ones
// BF16 copy of the weights in the workspace: W_1 .. W_4 each already in its
// K-major operand-tile layout (one bulk copy per tile; the tiles are contiguous
// in the forward's shared memory too), then w5
__host__ __device__ constexpr int wtile_off(int l) { return l == 1 ? 0 : kRows * kF * 2 + (l - 2) * kTileBytes; }
constexpr int kW5 = (kRows * kF * 2 + (kL - 1) * kTileBytes) / 2;   // bf16 index of w5
constexpr int kWbf = kW5 + kH;                // one copy (114,944 bytes, a multiple of 256)
// Every CTA reads the same weights: kWRep copies (CTA b reads copy b % kWRep)
// spread those reads over more L2 lines than one copy would.
constexpr int kWRep = 8;

struct NfArgs {
    int G;                 // nodes per side
    int rows;              // G * G
    float freqs[16];       // cycles per field of view
    float v_mid, v_half, v_bg;
    const float* params;   // [kNParam] FP32 master parameters
    const unsigned char* mask;   // [G*G] or NULL (all inside)
    __nv_bfloat16* wbf;    // [kWRep][kWbf] BF16 copies of the weights (workspace)
    unsigned char* htiles; // [cta][kL][kTileBytes] layer outputs in operand layout (workspace)
    float* t5;             // [rows] tanh of the output pre-activation (workspace)
    float* sos;            // [G*G] forward output
    const float* dL_dsos;  // backward input
    float* part;           // [cta][kPartStride] per-CTA parameter gradients (workspace)
    int* status;           // workspace word: set to 1 if a wait gave up
    unsigned long long limit_ns;   // bound on every wait (pact_set_wait_limit_ns)
};

// Features of node `row` written as row `r` of a K-major [128 x 64] tile.
__device__ __forceinline__ void features(const NfArgs& a, int row, float (&f)[kF]) {
    const int p = row / a.G, q = row - (row / a.G) * a.G;
    const float x = (q - 0.5f * (a.G - 1)) / a.G, y = (p - 0.5f * (a.G - 1)) / a.G;
#pragma unroll
    for (int l = 0; l < 16; ++l) {
        float sx, cx, sy, cy;
        sincospif(2.f * a.freqs[l] * x, &sx, &cx);
        sincospif(2.f * a.freqs[l] * y, &sy, &cy);
        f[4 * l + 0] = sx;
        f[4 * l + 1] = cx;
        f[4 * l + 2] = sy;
        f[4 * l + 3] = cy;
    }
}

__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}

// 8 consecutive K elements (one 16-byte core-matrix row) of row r at column k0.
__device__ __forceinline__ void st8(unsigned char* tile, int r, int k0, int K, const float* v) {
    uint4 u;
    u.x = pack2(v[0], v[1]);
    u.y = pack2(v[2], v[3]);
    u.z = pack2(v[4], v[5]);
    u.w = pack2(v[6], v[7]);
    *reinterpret_cast<uint4*>(tile + umma::kmaj_off(r, k0, K)) = u;
}


// Element u (0..7) of eight BF16 values packed in a uint4, as FP32 (a BF16 is
// the upper half of the FP32 with the same bits).
__device__ __forceinline__ float bf16_at(const uint4& v, int u) {
    const uint32_t w = u < 2 ? v.x : u < 4 ? v.y : u < 6 ? v.z : v.w;
    return __uint_as_float((u & 1) ? (w & 0xFFFF0000u) : (w << 16));
}

// 1-D bulk copy shared -> global in this thread's bulk group (16-byte aligned,
// bytes a multiple of 16), and the waits on this thread's bulk groups: until
// at most N are still reading shared memory, and until all have completed.
__device__ __forceinline__ void bulk_s2g(void* dst, const void* src, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_addr(src)),
                 "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void bulk_wait_read() {
    asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// Weight tile W_l (workspace, operand layout) -> dst by one bulk copy on `bar`.
__device__ __forceinline__ const __nv_bfloat16* my_wbf(const NfArgs& a) {
    return a.wbf + (size_t)(blockIdx.x % kWRep) * kWbf;
}
__device__ __forceinline__ void fetch_w(unsigned char* dst, const NfArgs& a, int l, uint64_t* bar) {
    tma_bulk_g2s(dst, reinterpret_cast<const unsigned char*>(my_wbf(a)) + wtile_off(l),
                 (uint32_t)(kH * in_dim(l) * 2), bar);
}

// Bounded mbarrier wait; a wait that gives up sets the status word.
__device__ __forceinline__ bool wait_bar(uint64_t* bar, uint32_t parity, int* status, unsigned long long limit) {
    const bool ok = mbar_wait_bounded(bar, parity, limit);
    if (!ok) atomicExch(status, 1);
    return ok;
}

// BF16 copies of the weights: eight consecutive elements (o, c .. c + 7) of
// W_l to their 16-byte row of the K-major [out x in] tile of layer l, w5 after
// the tiles (biases stay FP32).  One thread per eight weights.
constexpr int kCast8 = (kH * kF + (kL - 1) * kH * kH + kH) / 8;
__global__ void nf_cast_kernel(const float* params, __nv_bfloat16* wbf) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= kCast8) return;
    int src, dst;                                   // first parameter; destination in bytes
    if (t < kH * kF / 8) {                          // W_1: [128 x 64]
        const int o = t / (kF / 8), c = (t - o * (kF / 8)) * 8;
        src = off_w(1) + o * kF + c;
        dst = wtile_off(1) + (int)umma::kmaj_off(o, c, kF);
    } else if (t < kCast8 - kH / 8) {               // W_2 .. W_4: [128 x 128]
        const int u = t - kH * kF / 8, l = 2 + u / (kH * kH / 8), v = u - (l - 2) * (kH * kH / 8);
        const int o = v / (kH / 8), c = (v - o * (kH / 8)) * 8;
        src = off_w(l) + o * kH + c;
        dst = wtile_off(l) + (int)umma::kmaj_off(o, c, kH);
    } else {                                        // w5
        const int c = (t - (kCast8 - kH / 8)) * 8;
        src = kOffW5 + c;
        dst = 2 * (kW5 + c);
    }
    float v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = params[src + u];
    uint4 q;
    q.x = pack2(v[0], v[1]);
    q.y = pack2(v[2], v[3]);
    q.z = pack2(v[4], v[5]);
    q.w = pack2(v[6], v[7]);
#pragma unroll
    for (int r = 0; r < kWRep; ++r)
        *reinterpret_cast<uint4*>(reinterpret_cast<unsigned char*>(wbf + (size_t)r * kWbf) + dst) = q;
}

__global__ void __launch_bounds__(kRows, 1) nf_fwd_kernel(const NfArgs a) {
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char* A0 = sm;                                 // features  [128 x 64]   16 KB
    auto Hb = [](int i) { return sm + 16384 + i * kTileBytes; };            // layer outputs  2 x 32 KB
    unsigned char* Wt = sm + 16384 + 2 * kTileBytes;        // W1 (16 KB), W2..W4 (32 KB each), as in the workspace
    __shared__ __align__(16) float bias_s[kL][kH];
    __shared__ float w5_s[kH];
    __shared__ uint32_t tmem_s;
    __shared__ __align__(8) uint64_t bar, wbar[kL];
    __shared__ int wbad_s;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int row = blockIdx.x * kRows + tid;
    const bool valid = row < a.rows;

    if (tid == 0) {                                 // the four weight tiles, one bulk copy each
        mbar_init(&bar, 1);
        for (int l = 0; l < kL; ++l) mbar_init(&wbar[l], 1);
        mbar_init_fence();
        wbad_s = 0;
        for (int l = 1; l <= kL; ++l) {
            mbar_arrive_expect_tx(&wbar[l - 1], (uint32_t)(kH * in_dim(l) * 2));
            fetch_w(Wt + wtile_off(l), a, l, &wbar[l - 1]);
        }
    }
    for (int c = tid; c < kL * kH; c += blockDim.x) bias_s[c / kH][c % kH] = a.params[off_b(c / kH + 1) + c % kH];
    for (int c = tid; c < kH; c += blockDim.x) w5_s[c] = __bfloat162float(my_wbf(a)[kW5 + c]);
    {
        float f[kF];
        features(a, valid ? row : 0, f);
#pragma unroll
        for (int k0 = 0; k0 < kF; k0 += 8) st8(A0, tid, k0, kF, f + k0);
    }
    if (warp == 0) umma::tmem_alloc(&tmem_s, 128);
    umma::fence_smem_to_async();
    umma::fence_before();
    __syncthreads();
    umma::fence_after();
    const uint32_t tmem = tmem_s;
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
    bool ok = true;
    float z5p[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};   // independent partial sums of the head
    const float b5 = a.params[kOffB5];
    const bool inside = valid && (a.mask ? a.mask[row] != 0 : true);
    for (int l = 1; l <= kL; ++l) {
        const unsigned char* in = l == 1 ? A0 : Hb(l % 2);
        unsigned char* out = Hb((l + 1) % 2);
        const int K = in_dim(l);
        if (tid == 0) {
            if (!wait_bar(&wbar[l - 1], 0u, a.status, a.limit_ns)) wbad_s = 1;   // W_l has landed
            if (l >= 3) bulk_wait_read<1>();       // `out` (layer l - 2's output) has been read by its store
            for (int kk = 0; kk < K / 16; ++kk)
                umma::mma(tmem, umma::kslice(in, K, kk), umma::kslice(Wt + wtile_off(l), K, kk),
                          umma::idesc_bf16(128, 128), kk > 0);
            umma::commit(&bar);
        }
        ok = wait_bar(&bar, (uint32_t)((l - 1) & 1), a.status, a.limit_ns) && ok;
        umma::fence_after();
        for (int c0 = 0; c0 < kH; c0 += 64) {
            float v[64];
            umma::ld64(tmem + lane_base + c0, v);
#pragma unroll
            for (int j = 0; j < 64; j += 4) {
                const float4 b4 = *reinterpret_cast<const float4*>(&bias_s[l - 1][c0 + j]);
                v[j] = fmaxf(v[j] + b4.x, 0.f);
                v[j + 1] = fmaxf(v[j + 1] + b4.y, 0.f);
                v[j + 2] = fmaxf(v[j + 2] + b4.z, 0.f);
                v[j + 3] = fmaxf(v[j + 3] + b4.w, 0.f);
            }
            if (l == kL) {                          // the head sees the BF16 values the tile holds
#pragma unroll
                for (int j = 0; j < 64; ++j)
                    z5p[j & 7] = fmaf(__bfloat162float(__float2bfloat16_rn(v[j])), w5_s[c0 + j], z5p[j & 7]);
            }
#pragma unroll
            for (int j = 0; j < 64; j += 8) st8(out, tid, c0 + j, kH, v + j);
        }
        umma::fence_smem_to_async();
        umma::fence_before();
        __syncthreads();
        umma::fence_after();
        // layer output tile (operand layout) to the workspace for the backward pass,
        // by one bulk copy that runs on while the next layer computes
        if (tid == 0) bulk_s2g(a.htiles + ((size_t)blockIdx.x * kL + (l - 1)) * kTileBytes, out, kTileBytes);
    }
    ok = ok && !wbad_s;                             // (set before the last layer's barrier)
    const float z5 = ((z5p[0] + z5p[1]) + (z5p[2] + z5p[3])) + ((z5p[4] + z5p[5]) + (z5p[6] + z5p[7]));
    const float t = tanhf(z5 + b5);
    if (valid) {
        a.t5[row] = ok ? t : __int_as_float(0x7fc00000);
        a.sos[row] = inside ? (ok ? fmaf(a.v_half, t, a.v_mid) : __int_as_float(0x7fc00000)) : a.v_bg;
    }
    if (tid == 0) {
        bulk_wait_all();                            // the tiles are in the workspace
        if (wbad_s)                                 // a weight copy gave up: let it land before the CTA ends
            for (int l = 0; l < kL; ++l) mbar_wait_bounded(&wbar[l], 0u, a.limit_ns);
    }
    umma::fence_before();
    __syncthreads();
    if (warp == 0) umma::tmem_dealloc(tmem, 128);
}

__global__ void __launch_bounds__(kRows, 1) nf_bwd_kernel(const NfArgs a) {
    extern __shared__ __align__(1024) unsigned char sm[];
    // dz and h_{l-1} are K-major tiles [nodes x units]; read as MN-major they
    // are the transposed operands dz^T and h^T of the weight-gradient GEMM
    // Layer l reads h_{l-1} and W_l from buffers l & 1; the copies for layer l - 1
    // go into the other pair while layer l runs (the pair layer l + 1 has finished with).
    unsigned char* dzA = sm;                      // dz         [128 nodes x out]    32 KB
    auto Hb = [](int i) { return sm + (1 + i) * kTileBytes; };   // h_{l-1} [128 nodes x in]  2 x 32 KB
    auto Wb = [](int i) { return sm + (3 + i) * kTileBytes; };   // W_l     [out x in]        2 x 32 KB
    unsigned char* ones = sm + 5 * kTileBytes;    // [16 x 128 nodes] of 1.0: db = dz^T 1 on the tensor core   4 KB
    unsigned char* gsplit = ones + kOnesBytes;    // [16 x 128 nodes]: rows 0, 1 = g5 as BF16 high part + remainder  4 KB
    __shared__ float w5_s[kH];
    __shared__ float red_s[kRows / 32];
    __shared__ uint32_t tmem_s;
    // bbar[i]: bulk copies into the buffer pair (Hb(i), Wb(i)); bbar[1] phase 0
    // is h4 alone, then each pair is filled for one layer at a time
    __shared__ __align__(8) uint64_t bar, bbar[2];
    const int tid = threadIdx.x, warp = tid >> 5;
    const int row = blockIdx.x * kRows + tid;
    const bool valid = row < a.rows;
    float* part = a.part + (size_t)blockIdx.x * kPartStride;   // 16-byte aligned rows for float4 stores
    const unsigned char* tiles = a.htiles + (size_t)blockIdx.x * kL * kTileBytes;

    // output layer: g5 = dL/dv dv/dz = dL/dv v_half (1 - t^2), inside the mask
    float g5 = 0.f;
    if (valid && (a.mask ? a.mask[row] != 0 : true)) {
        const float t = a.t5[row];
        g5 = a.dL_dsos[row] * a.v_half * (1.f - t * t);
    }
    // h4 of this CTA (operand layout) -> Hb(1); then layer kL's h3 and W4 -> Hb(0), Wb(0);
    // one bulk copy per tile
    unsigned char* H4 = Hb(1);
    if (tid == 0) {
        mbar_init(&bar, 1);
        mbar_init(&bbar[0], 1);
        mbar_init(&bbar[1], 1);
        mbar_init_fence();
        mbar_arrive_expect_tx(&bbar[1], kTileBytes);
        tma_bulk_g2s(H4, tiles + (size_t)(kL - 1) * kTileBytes, kTileBytes, &bbar[1]);
        mbar_arrive_expect_tx(&bbar[0], 2 * kTileBytes);
        tma_bulk_g2s(Hb(kL & 1), tiles + (size_t)(kL - 2) * kTileBytes, kTileBytes, &bbar[0]);
        fetch_w(Wb(kL & 1), a, kL, &bbar[0]);
    }
    for (int c = tid; c < kOnesBytes / 16; c += blockDim.x)
        reinterpret_cast<uint4*>(ones)[c] = make_uint4(0x3F803F80u, 0x3F803F80u, 0x3F803F80u, 0x3F803F80u);
    if (warp == 0) umma::tmem_alloc(&tmem_s, 512);
    w5_s[tid] = __bfloat162float(my_wbf(a)[kW5 + tid]);
    __syncthreads();
    bool ok = wait_bar(&bbar[1], 0u, a.status, a.limit_ns);   // h4 has landed
    // dz4 = g5 w5 (h4 > 0) for this node
#pragma unroll 1
    for (int c = 0; c < kH; c += 8) {
        const uint4 hv = *reinterpret_cast<const uint4*>(H4 + umma::kmaj_off(tid, c, kH));
        float dz[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) dz[u] = bf16_at(hv, u) > 0.f ? g5 * w5_s[c + u] : 0.f;
        st8(dzA, tid, c, kH, dz);
    }
    // dW5 = h4^T g5 on the tensor core: g5 split into a BF16 high part and the
    // BF16 remainder (rows 0 and 1 of a [16 x nodes] tile; together about 16
    // significant bits), the two result columns added in FP32
    {
        const __nv_bfloat16 hi = __float2bfloat16_rn(g5);
        const __nv_bfloat16 lo = __float2bfloat16_rn(g5 - __bfloat162float(hi));
        const __nv_bfloat16 zero = __float2bfloat16_rn(0.f);
#pragma unroll
        for (int n = 0; n < 16; ++n)
            *reinterpret_cast<__nv_bfloat16*>(gsplit + umma::kmaj_off(n, tid, kRows)) = n == 0 ? hi : (n == 1 ? lo : zero);
    }
    umma::fence_smem_to_async();
    umma::fence_before();
    __syncthreads();
    umma::fence_after();
    if (tid == 0) {
        for (int kk = 0; kk < kRows / 16; ++kk)
            umma::mma(tmem_s + 256, umma::mn_slice(H4, kH, kk), umma::kslice(gsplit, kRows, kk),
                      umma::idesc_bf16(128, 16) | (1u << 15), kk > 0);
        umma::commit(&bar);
    }
    // db5 = sum over nodes of g5, a fixed-order block reduction
    {
        const float b = warp_sum(g5);
        if ((tid & 31) == 0) red_s[warp] = b;
    }
    wait_bar(&bar, 0u, a.status, a.limit_ns);
    umma::fence_after();
    {
        const uint32_t lb = (uint32_t)(warp * 32) << 16;
        part[kOffW5 + tid] = umma::ld1(tmem_s + 256 + lb) + umma::ld1(tmem_s + 257 + lb);
    }
    if (tid == 0) {
        float b = 0.f;
        for (int w = 0; w < kRows / 32; ++w) b += red_s[w];
        part[kOffB5] = b;
    }
    umma::fence_before();
    __syncthreads();
    umma::fence_after();

    const uint32_t tmem = tmem_s;
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
    uint32_t phase = 1;                             // phase 0 was the dW5 product
    for (int l = kL; l >= 1; --l) {
        const int K_in = in_dim(l);
        unsigned char* Hr = Hb(l & 1);
        unsigned char* WT = Wb(l & 1);
        // copies for layer l - 1 (h_{l-2}, W_{l-1}) into the other pair (read by layer
        // l + 1, finished), then wait for layer l's
        if (l - 1 >= 2 && tid == 0) {
            fence_proxy_async_smem();
            uint64_t* nb = &bbar[(l - 1) & 1];
            mbar_arrive_expect_tx(nb, 2 * kTileBytes);
            tma_bulk_g2s(Hb((l - 1) & 1), tiles + (size_t)(l - 3) * kTileBytes, kTileBytes, nb);
            fetch_w(Wb((l - 1) & 1), a, l - 1, nb);   // W [out x in] K-major = W^T read MN-major
        }
        if (l > 1) {                                // h_{l-1} and W_l have landed
            ok = wait_bar(&bbar[l & 1], l < kL ? 1u : 0u, a.status, a.limit_ns) && ok;
        } else {
            float f[kF];
            features(a, valid ? row : 0, f);
#pragma unroll
            for (int k0 = 0; k0 < kF; k0 += 8) st8(Hr, tid, k0, kF, f + k0);
        }
        umma::fence_smem_to_async();
        umma::fence_before();
        __syncthreads();
        umma::fence_after();
        if (tid == 0) {
            // dW_l [out x in] = dz^T [out x nodes] * (h^T [in x nodes])^T, both operands
            // the K-major node tiles read MN-major (M = out, N = in, K = nodes)
            for (int kk = 0; kk < kRows / 16; ++kk)
                umma::mma(tmem, umma::mn_slice(dzA, kH, kk), umma::mn_slice(Hr, K_in, kk),
                          umma::idesc_bf16_mn(128, K_in), kk > 0);
            // dh_{l-1} [nodes x in] = dz [nodes x out] * (W^T [in x out])^T
            if (l > 1)
                for (int kk = 0; kk < kH / 16; ++kk)
                    umma::mma(tmem + 128, umma::kslice(dzA, kH, kk), umma::mn_slice(WT, kH, kk),
                              umma::idesc_bf16(128, kH) | (1u << 16), kk > 0);
            // db_l [out x 16] = dz^T [out x nodes] * (ones [16 x nodes])^T: every column is the sum over nodes
            for (int kk = 0; kk < kRows / 16; ++kk)
                umma::mma(tmem + 256, umma::mn_slice(dzA, kH, kk), umma::kslice(ones, kRows, kk),
                          umma::idesc_bf16(128, 16) | (1u << 15), kk > 0);
            umma::commit(&bar);
        }
        wait_bar(&bar, phase, a.status, a.limit_ns);
        phase ^= 1u;
        umma::fence_after();
        part[off_b(l) + tid] = umma::ld1(tmem + 256 + lane_base);   // db_l[tid]
        // weight-gradient row `tid` (TMEM lane = output unit), stored as [in/4][out][4]
        // so that a warp's float4 stores are 512 contiguous bytes
        for (int c0 = 0; c0 < K_in; c0 += 64) {
            float v[64];
            umma::ld64(tmem + lane_base + c0, v);
            float4* dst = reinterpret_cast<float4*>(part + off_w(l)) + tid;
#pragma unroll
            for (int j = 0; j < 64; j += 4) dst[((c0 + j) >> 2) * kH] = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
        }
        if (l > 1) {
            // dz_{l-1} = dh (h_{l-1} > 0), node `tid`
            for (int c0 = 0; c0 < kH; c0 += 64) {
                float v[64];
                umma::ld64(tmem + 128 + lane_base + c0, v);
#pragma unroll
                for (int j = 0; j < 64; j += 8) {
                    const uint4 hv = *reinterpret_cast<const uint4*>(Hr + umma::kmaj_off(tid, c0 + j, kH));
                    float dz[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) dz[u] = bf16_at(hv, u) > 0.f ? v[j + u] : 0.f;
                    st8(dzA, tid, c0 + j, kH, dz);
                }
            }
        }
        umma::fence_before();
        __syncthreads();
        umma::fence_after();
    }
    if (!ok) part[off_b(1) + tid] = __int_as_float(0x7fc00000);   // a copy never landed: poison the gradient
    if (tid == 0 && !ok)                            // and let the copies in flight land before the CTA ends
        for (int i = 0; i < 2; ++i) mbar_wait_bounded(&bbar[i], 1u, a.limit_ns);
    umma::fence_before();
    __syncthreads();
    if (warp == 0) umma::tmem_dealloc(tmem, 512);
}

// Parameter index of slot q of a per-CTA gradient row: each weight block is
// stored as [in/4][out][4] (the backward's coalesced stores from TMEM rows),
// biases, w5 and b5 in parameter order.
__device__ __forceinline__ int param_of_slot(int q) {
#pragma unroll
    for (int l = 1; l <= kL; ++l)
        if (q >= off_w(l) && q < off_b(l)) {
            const int r = q - off_w(l);
            return off_w(l) + ((r >> 2) & (kH - 1)) * in_dim(l) + 4 * (r >> 9) + (r & 3);
        }
    return q;
}

// dL/dparams = sum over CTAs of the per-CTA rows, in a fixed order; one thread
// per row slot (coalesced reads, sixteen in flight), written to its parameter.
__global__ void __launch_bounds__(128) nf_reduce_kernel(const float* part, int nct, float* out, int accumulate) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= kNParam) return;
    float s[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) s[u] = 0.f;
    int c = 0;
    for (; c + 16 <= nct; c += 16) {
        float v[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) v[u] = __ldcg(part + (size_t)(c + u) * kPartStride + q);
#pragma unroll
        for (int u = 0; u < 16; ++u) s[u] += v[u];
    }
    for (; c < nct; ++c) s[0] += part[(size_t)c * kPartStride + q];
#pragma unroll
    for (int w = 8; w > 0; w >>= 1)
#pragma unroll
        for (int u = 0; u < w; ++u) s[u] += s[u + w];
    const float t = s[0];
    const int p = param_of_slot(q);
    out[p] = accumulate ? out[p] + t : t;
}

struct NfPlan {
    int rows, nct;
    size_t off_htiles, off_t5, off_part, off_status, total;
    size_t smem_fwd, smem_bwd;
};

NfPlan nf_plan(const pact_geometry* g) {
    NfPlan p;
    p.rows = g->sos_g * g->sos_g;
    p.nct = (p.rows + kRows - 1) / kRows;
    size_t o = align_up((size_t)kWRep * kWbf * sizeof(__nv_bfloat16), 256);
    p.off_htiles = o;
    o += align_up((size_t)p.nct * kL * kTileBytes, 256);
    p.off_t5 = o;
    o += align_up((size_t)p.rows * sizeof(float), 256);
    p.off_part = o;
    o += align_up((size_t)p.nct * kPartStride * sizeof(float), 256);
    p.off_status = o;
    o += 256;
    p.total = o;
    p.smem_fwd = 16384 + 2 * kTileBytes + 16384 + (kL - 1) * kTileBytes;
    p.smem_bwd = 5 * kTileBytes + 2 * kOnesBytes;
    return p;
}

pact_status nf_args(const pact_geometry* g, const float* params, const unsigned char* mask, float v_mid,
                    float v_half, void* ws, size_t ws_bytes, NfArgs& a, NfPlan& pl) {
    PACT_TRY(check_geometry(g));
    if (!params) return fail(PACT_ERR_INVALID_ARG, "nf: params is NULL");
    if (!ws) return fail(PACT_ERR_INVALID_ARG, "nf: workspace is NULL");
    if (reinterpret_cast<uintptr_t>(ws) % 256) return fail(PACT_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    if (reinterpret_cast<uintptr_t>(params) % 16) return fail(PACT_ERR_INVALID_ARG, "nf: params must be 16-byte aligned");
    if (!(v_half > 0.f)) return fail(PACT_ERR_INVALID_ARG, "nf: v_half must be > 0");
    pl = nf_plan(g);
    if (ws_bytes < pl.total) return fail(PACT_ERR_INVALID_ARG, "nf: workspace too small: %zu < %zu bytes", ws_bytes, pl.total);
    char* base = static_cast<char*>(ws);
    a.G = g->sos_g;
    a.rows = pl.rows;
    for (int l = 0; l < 16; ++l) a.freqs[l] = (float)pow(64.0, l / 15.0);
    a.v_mid = v_mid;
    a.v_half = v_half;
    a.v_bg = g->v_bg;
    a.params = params;
    a.mask = mask;
    a.wbf = reinterpret_cast<__nv_bfloat16*>(base);
    a.htiles = reinterpret_cast<unsigned char*>(base + pl.off_htiles);
    a.t5 = reinterpret_cast<float*>(base + pl.off_t5);
    a.part = reinterpret_cast<float*>(base + pl.off_part);
    a.status = reinterpret_cast<int*>(base + pl.off_status);
    a.limit_ns = wait_limit_ns();
    a.sos = nullptr;
    a.dL_dsos = nullptr;
    return PACT_OK;
}

}  // namespace
}  // namespace pact

using namespace pact;

extern "C" int pact_nf_param_count(void) { return kNParam; }

extern "C" size_t pact_nf_workspace_size(const pact_geometry* g) {
    if (check_geometry(g) != PACT_OK) return 0;
    return nf_plan(g).total;
}

extern "C" pact_status pact_nf_forward(const pact_geometry* g, const float* params, const unsigned char* mask,
                                       float v_mid, float v_half, float* sos, void* ws, size_t ws_bytes,
                                       void* stream) {
    NfArgs a;
    NfPlan pl;
    PACT_TRY(nf_args(g, params, mask, v_mid, v_half, ws, ws_bytes, a, pl));
    if (!sos) return fail(PACT_ERR_INVALID_ARG, "nf_forward: sos is NULL");
    a.sos = sos;
    cudaStream_t st = as_stream(stream);
    if (cudaMemsetAsync(a.status, 0, sizeof(int), st) != cudaSuccess) return check_launch("nf_forward: memset");
    nf_cast_kernel<<<(kCast8 + 255) / 256, 256, 0, st>>>(params, a.wbf);
    PACT_TRY(check_launch("nf_forward: weight cast"));
    PACT_TRY(ensure_smem((const void*)nf_fwd_kernel, pl.smem_fwd, "nf_forward: shared memory attribute"));
    nf_fwd_kernel<<<pl.nct, kRows, pl.smem_fwd, st>>>(a);
    return check_launch("nf_forward kernel");
}

extern "C" pact_status pact_nf_backward(const pact_geometry* g, const float* params, const unsigned char* mask,
                                        float v_mid, float v_half, const float* dL_dsos, float* dL_dparams,
                                        int accumulate, void* ws, size_t ws_bytes, void* stream) {
    NfArgs a;
    NfPlan pl;
    PACT_TRY(nf_args(g, params, mask, v_mid, v_half, ws, ws_bytes, a, pl));
    if (!dL_dsos || !dL_dparams) return fail(PACT_ERR_INVALID_ARG, "nf_backward: dL_dsos and dL_dparams must not be NULL");
    a.dL_dsos = dL_dsos;
    cudaStream_t st = as_stream(stream);
    PACT_TRY(ensure_smem((const void*)nf_bwd_kernel, pl.smem_bwd, "nf_backward: shared memory attribute"));
    nf_bwd_kernel<<<pl.nct, kRows, pl.smem_bwd, st>>>(a);
    PACT_TRY(check_launch("nf_backward kernel"));
    nf_reduce_kernel<<<(kNParam + 127) / 128, 128, 0, st>>>(a.part, pl.nct, dL_dparams, accumulate);
    return check_launch("nf_backward reduction");
}

extern "C" pact_status pact_nf_status(const pact_geometry* g, const void* ws, size_t ws_bytes, int* host_status,
                                      void* stream) {
    PACT_TRY(check_geometry(g));
    if (!ws || !host_status) return fail(PACT_ERR_INVALID_ARG, "nf_status: null pointer");
    const NfPlan pl = nf_plan(g);
    if (ws_bytes < pl.total) return fail(PACT_ERR_INVALID_ARG, "nf_status: workspace too small");
    cudaStream_t st = as_stream(stream);
    if (cudaMemcpyAsync(host_status, static_cast<const char*>(ws) + pl.off_status, sizeof(int),
                        cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return check_launch("nf_status: copy");
    return *host_status ? fail(PACT_ERR_TIMEOUT, "nf: a tensor-core completion wait gave up") : PACT_OK;
}
