// Checkerboard Gibbs sampling of the square-lattice Ising model (§4.3.1).
//
// Spins s_i in {0, 1}, 4-neighbour lattice with free boundary, conditional
// P(s_i = 1 | rest) = 1 / (1 + exp(-z_i)) with z_i = b_i + w * (sum of the
// neighbours' spins). The two colours of the checkerboard (colour c: sites
// with (row + col) % 2 == c) are conditionally independent, so a half-sweep
// updates a whole colour at once; a sweep is colour 0 then colour 1. As the
// paper does for vectorisation, each colour lives in its own dense "plane"
// (plane entry (r, j) is the site (r, 2j + (r + c) % 2)), so every access is
// unit-stride, and the uniforms arrive as a batch (§4.3.1, batch RNG).
//
// In plane terms the neighbours of colour-c entry (r, j), all in the other
// plane: (r - 1, j), (r + 1, j), and in row r the entries j - 1 + o and j + o,
// o = (r + c) % 2. One thread updates 8 consecutive entries of a row: it
// reads 8 biases and 8 uniforms (float4 loads), 8 bytes of each of the
// other plane's rows r - 1, r, r + 1 and the two bytes beyond the middle
// row's ends, and writes 8 bytes of spins. Neighbours outside the lattice
// read as 0, which is the free boundary. (8 rather than 16 entries per
// thread: 40 instead of 50 registers, more resident warps and loads in
// flight; measured 105 against 148 µs per 8192 x 8192 sweep.)
#include <cstring>

#include "glm_internal.cuh"

namespace glm {

constexpr int kIsingChunk = 8;           // plane entries per thread (8 or 16 supported)
constexpr int kIsingThreads = 256;

struct IsingParams {
    uint8_t *s_c;              // plane being updated
    const uint8_t *s_o;        // the other plane
    const float *b_c;          // biases of the updated plane
    const float *u;            // uniforms of this half-sweep (plane order)
    int rows;
    int H;                     // entries per plane row (cols / 2)
    int color;
    float w;
    unsigned long long *ones;  // count of 1s in the updated plane, or null
    int fast;                  // H % 16 == 0 and 16-byte aligned planes
};

namespace is {

template <int W>
__device__ __forceinline__ int byte_of(const uint32_t (&v)[W], int t)
{
    return (int)((v[t >> 2] >> (8 * (t & 3))) & 0xFFu);
}

// W 32-bit words of spins (W = 4: one 16-byte load, W = 2: one 8-byte load;
// the vector path keeps rows chunk-aligned)
template <int W>
__device__ __forceinline__ void load_words(const uint8_t *p, uint32_t (&v)[W])
{
    if constexpr (W == 4) {
        const uint4 x = *reinterpret_cast<const uint4 *>(p);
        v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
    } else {
        const uint2 x = *reinterpret_cast<const uint2 *>(p);
        v[0] = x.x; v[1] = x.y;
    }
}

template <int W>
__device__ __forceinline__ void store_words(uint8_t *p, const uint32_t (&v)[W])
{
    if constexpr (W == 4)
        *reinterpret_cast<uint4 *>(p) = make_uint4(v[0], v[1], v[2], v[3]);
    else
        *reinterpret_cast<uint2 *>(p) = make_uint2(v[0], v[1]);
}

__device__ __forceinline__ uint8_t decide(float b, float w, int n, float u)
{
    const float z = fmaf(w, (float)n, b);
    const float p = __fdividef(1.0f, 1.0f + __expf(-z));
    return u < p ? 1 : 0;
}

}  // namespace is

__global__ void __launch_bounds__(kIsingThreads) ising_half_kernel(IsingParams p)
{
    const int cpr = (p.H + kIsingChunk - 1) / kIsingChunk;     // chunks per row
    const int64_t nchunks = (int64_t)p.rows * cpr;
    unsigned cnt = 0;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nchunks;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(q / cpr);
        const int j0 = (int)(q - (int64_t)r * cpr) * kIsingChunk;
        const int o = (r + p.color) & 1;
        const int64_t row = (int64_t)r * p.H;
        if (p.fast) {
            constexpr int CH = kIsingChunk, W = CH / 4;
            const float4 *bp = reinterpret_cast<const float4 *>(p.b_c + row + j0);
            const float4 *up = reinterpret_cast<const float4 *>(p.u + row + j0);
            float bv[CH], uv[CH];
#pragma unroll
            for (int v = 0; v < CH / 4; ++v) {
                const float4 x = __ldcs(bp + v);
                const float4 y = __ldcs(up + v);
                bv[4 * v] = x.x; bv[4 * v + 1] = x.y; bv[4 * v + 2] = x.z; bv[4 * v + 3] = x.w;
                uv[4 * v] = y.x; uv[4 * v + 1] = y.y; uv[4 * v + 2] = y.z; uv[4 * v + 3] = y.w;
            }
            uint32_t mid[W], above[W], below[W];
            is::load_words<W>(p.s_o + row + j0, mid);
#pragma unroll
            for (int v = 0; v < W; ++v)
                above[v] = below[v] = 0u;
            if (r > 0)
                is::load_words<W>(p.s_o + row - p.H + j0, above);
            if (r + 1 < p.rows)
                is::load_words<W>(p.s_o + row + p.H + j0, below);
            const int le = j0 > 0 ? p.s_o[row + j0 - 1] : 0;
            const int re = j0 + CH < p.H ? p.s_o[row + j0 + CH] : 0;
            uint32_t outw[W];
#pragma unroll
            for (int v = 0; v < W; ++v)
                outw[v] = 0u;
#pragma unroll
            for (int t = 0; t < CH; ++t) {
                // row-r neighbours: entries t - 1 + o and t + o of the chunk
                const int left = o ? is::byte_of<W>(mid, t) : (t == 0 ? le : is::byte_of<W>(mid, t - 1));
                const int right = o ? (t == CH - 1 ? re : is::byte_of<W>(mid, t + 1)) : is::byte_of<W>(mid, t);
                const int n = left + right + is::byte_of<W>(above, t) + is::byte_of<W>(below, t);
                const uint8_t sv = is::decide(bv[t], p.w, n, uv[t]);
                outw[t >> 2] |= (uint32_t)sv << (8 * (t & 3));
                cnt += sv;
            }
            is::store_words<W>(p.s_c + row + j0, outw);
        } else {
            const int j1 = j0 + kIsingChunk < p.H ? j0 + kIsingChunk : p.H;
            for (int j = j0; j < j1; ++j) {
                const int li = j - 1 + o, ri = j + o;
                const int left = li >= 0 ? p.s_o[row + li] : 0;
                const int right = ri < p.H ? p.s_o[row + ri] : 0;
                const int above = r > 0 ? p.s_o[row - p.H + j] : 0;
                const int below = r + 1 < p.rows ? p.s_o[row + p.H + j] : 0;
                const uint8_t sv = is::decide(p.b_c[row + j], p.w, left + right + above + below,
                                              p.u[row + j]);
                p.s_c[row + j] = sv;
                cnt += sv;
            }
        }
    }
    if (p.ones) {
#pragma unroll
        for (int m = 16; m > 0; m >>= 1)
            cnt += __shfl_xor_sync(0xFFFFFFFFu, cnt, m);
        if ((threadIdx.x & 31) == 0 && cnt)
            atomicAdd(p.ones, (unsigned long long)cnt);
    }
}

// natural layout <-> colour planes, elem_bytes 1 or 4
template <typename T>
__global__ void ising_split_kernel(const T *__restrict__ nat, int rows, int cols, T *__restrict__ p0,
                                   T *__restrict__ p1)
{
    const int64_t total = (int64_t)rows * cols;
    const int H = cols / 2;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(i / cols);
        const int c = (int)(i - (int64_t)r * cols);
        T *dst = ((r + c) & 1) ? p1 : p0;
        dst[(int64_t)r * H + (c >> 1)] = nat[i];
    }
}

template <typename T>
__global__ void ising_merge_kernel(const T *__restrict__ p0, const T *__restrict__ p1, int rows, int cols,
                                   T *__restrict__ nat)
{
    const int64_t total = (int64_t)rows * cols;
    const int H = cols / 2;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(i / cols);
        const int c = (int)(i - (int64_t)r * cols);
        const T *src = ((r + c) & 1) ? p1 : p0;
        nat[i] = src[(int64_t)r * H + (c >> 1)];
    }
}

static int sm_count_now()
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess)
        return 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

static bool al16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace glm

using namespace glm;

extern "C" {

glm_status_t glm_ising_split(const void *nat, int32_t elem_bytes, int32_t rows, int32_t cols,
                             void *plane0, void *plane1, glm_stream_t stream)
{
    if (!nat || !plane0 || !plane1 || rows < 1 || cols < 2 || (cols & 1) ||
        (elem_bytes != 1 && elem_bytes != 4))
        return GLM_ERR_INVALID_ARG;
    const int sms = sm_count_now();
    if (sms == 0) {
        cudaGetLastError();
        return GLM_ERR_NO_DEVICE;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int64_t total = (int64_t)rows * cols;
    const int blocks = (int)((total + 255) / 256 < sms * 8 ? (total + 255) / 256 : sms * 8);
    if (elem_bytes == 1)
        ising_split_kernel<uint8_t><<<blocks, 256, 0, st>>>(static_cast<const uint8_t *>(nat), rows, cols,
                                                            static_cast<uint8_t *>(plane0),
                                                            static_cast<uint8_t *>(plane1));
    else
        ising_split_kernel<float><<<blocks, 256, 0, st>>>(static_cast<const float *>(nat), rows, cols,
                                                          static_cast<float *>(plane0),
                                                          static_cast<float *>(plane1));
    return cudaGetLastError() == cudaSuccess ? GLM_OK : GLM_ERR_CUDA;
}

glm_status_t glm_ising_merge(const void *plane0, const void *plane1, int32_t elem_bytes, int32_t rows,
                             int32_t cols, void *nat, glm_stream_t stream)
{
    if (!nat || !plane0 || !plane1 || rows < 1 || cols < 2 || (cols & 1) ||
        (elem_bytes != 1 && elem_bytes != 4))
        return GLM_ERR_INVALID_ARG;
    const int sms = sm_count_now();
    if (sms == 0) {
        cudaGetLastError();
        return GLM_ERR_NO_DEVICE;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int64_t total = (int64_t)rows * cols;
    const int blocks = (int)((total + 255) / 256 < sms * 8 ? (total + 255) / 256 : sms * 8);
    if (elem_bytes == 1)
        ising_merge_kernel<uint8_t><<<blocks, 256, 0, st>>>(static_cast<const uint8_t *>(plane0),
                                                            static_cast<const uint8_t *>(plane1), rows, cols,
                                                            static_cast<uint8_t *>(nat));
    else
        ising_merge_kernel<float><<<blocks, 256, 0, st>>>(static_cast<const float *>(plane0),
                                                          static_cast<const float *>(plane1), rows, cols,
                                                          static_cast<float *>(nat));
    return cudaGetLastError() == cudaSuccess ? GLM_OK : GLM_ERR_CUDA;
}

glm_status_t glm_ising_sweeps(uint8_t *s0, uint8_t *s1, const float *b0, const float *b1, int32_t rows,
                              int32_t cols, float w, int32_t n_sweeps, const float *u,
                              int64_t *ones_out, glm_stream_t stream)
{
    if (!s0 || !s1 || !b0 || !b1 || rows < 1 || cols < 2 || (cols & 1) || n_sweeps < 0 ||
        (n_sweeps > 0 && !u) || !(w == w) || (ones_out && (reinterpret_cast<uintptr_t>(ones_out) & 7u)))
        return GLM_ERR_INVALID_ARG;
    if (n_sweeps == 0)
        return GLM_OK;
    const int sms = sm_count_now();
    if (sms == 0) {
        cudaGetLastError();
        return GLM_ERR_NO_DEVICE;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int H = cols / 2;
    const int64_t plane = (int64_t)rows * H;
    if (ones_out && cudaMemsetAsync(ones_out, 0, sizeof(int64_t) * 2 * (size_t)n_sweeps, st) != cudaSuccess)
        return GLM_ERR_CUDA;
    // the vector path needs whole chunks per row (then float rows are 32-byte
    // and spin rows 8-byte aligned) and 16-byte aligned base pointers
    const bool fast = (H % kIsingChunk) == 0 && al16(s0) && al16(s1) && al16(b0) && al16(b1) && al16(u);
    const int64_t chunks = (int64_t)rows * ((H + kIsingChunk - 1) / kIsingChunk);
    int blocks = (int)((chunks + kIsingThreads - 1) / kIsingThreads);
    if (blocks > sms * 16)
        blocks = sms * 16;
    IsingParams p;
    std::memset(&p, 0, sizeof(p));
    p.rows = rows;
    p.H = H;
    p.w = w;
    p.fast = fast ? 1 : 0;
    for (int t = 0; t < n_sweeps; ++t) {
        for (int c = 0; c < 2; ++c) {
            p.s_c = c ? s1 : s0;
            p.s_o = c ? s0 : s1;
            p.b_c = c ? b1 : b0;
            p.u = u + ((int64_t)t * 2 + c) * plane;
            p.color = c;
            p.ones = ones_out ? reinterpret_cast<unsigned long long *>(ones_out + 2 * t + c) : nullptr;
            ising_half_kernel<<<blocks, kIsingThreads, 0, st>>>(p);
        }
    }
    return cudaGetLastError() == cudaSuccess ? GLM_OK : GLM_ERR_CUDA;
}

}  // extern "C"
