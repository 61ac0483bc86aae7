// k_sort.cu -- chain bookkeeping and the locality sort of whole chains.
//
// Chains are maximal runs of bonded beads; their membership never changes, so
// they are numbered once (in tag order) when the state is loaded.  A sort
// orders chains by the brick-major cell key of their first bead (bricks of
// 8^3 cells, x fastest inside and across bricks), ties by the tag of the first
// bead, and then moves every bead of every chain in one gather.  The result is
// a deterministic function of the positions: the atomics only fill buckets,
// and each bucket is then ranked by tag.
#include "hpf_internal.cuh"

namespace hpf {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;
constexpr int kBrick = 8;

// ------------------------------------------------------------------ scan

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* sh,
                                                         uint32_t& total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[warp] = x;
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        uint32_t w = lane < nw ? sh[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < nw) sh[lane] = w;  // inclusive warp totals
    }
    __syncthreads();
    total = sh[(blockDim.x >> 5) - 1];
    const uint32_t before = warp > 0 ? sh[warp - 1] : 0u;
    __syncthreads();
    return before + x - v;
}

// Exclusive scan of one tile of kScanTile items; tile total to sums[tile].
__global__ void __launch_bounds__(kScanThreads) k_scan_tiles(const uint32_t* in, uint32_t* out,
                                                             uint32_t* sums, long long L) {
    __shared__ uint32_t sh[32];
    const long long base = (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kScanItems;
    uint32_t v[kScanItems];
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = (base + k < L) ? in[base + k] : 0u;
        s += v[k];
    }
    uint32_t total;
    uint32_t run = block_exclusive_scan(s, sh, total);
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < L) out[base + k] = run;
        run += v[k];
    }
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void k_scan_add(uint32_t* out, const uint32_t* offs, long long L) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < L) out[i] += offs[i / kScanTile];
}

long long scan_scratch_words(long long L) {
    long long w = 0;
    while (L > 1) {
        L = (L + kScanTile - 1) / kScanTile;
        w += L + 1;
    }
    return w + 1;
}

// out[i] = sum_{j<i} in[i]; in == out allowed.  Returns the number of kernels.
int scan_exclusive(const uint32_t* in, uint32_t* out, long long L, uint32_t* scratch,
                   cudaStream_t s) {
    if (L <= 0) return 0;
    const long long tiles = (L + kScanTile - 1) / kScanTile;
    uint32_t* sums = scratch;
    k_scan_tiles<<<(unsigned)tiles, kScanThreads, 0, s>>>(in, out, sums, L);
    int launched = 1;
    if (tiles > 1) {
        launched += scan_exclusive(sums, sums, tiles, scratch + tiles + 1, s);
        k_scan_add<<<(unsigned)((L + 255) / 256), 256, 0, s>>>(out, sums, L);
        ++launched;
    }
    return launched;
}

// ------------------------------------------------------------------ chains

__global__ void k_heads(const uint32_t* __restrict__ meta, int n, uint32_t* __restrict__ hd) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) hd[i] = (meta[i] & kBondPrev) ? 0u : 1u;
}

// hx = exclusive scan of the head flags: chain id of bead i = hx[i] (head) or hx[i] - 1.
__global__ void k_chain_build(const uint32_t* __restrict__ meta, const uint32_t* __restrict__ hx,
                              int n, int* __restrict__ cstart, uint32_t* __restrict__ tag0,
                              int* __restrict__ chain_of) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t m = meta[i];
    const bool head = !(m & kBondPrev);
    const int c = (int)hx[i] - (head ? 0 : 1);
    chain_of[i] = c;
    if (head) {
        cstart[c] = i;
        tag0[c] = m & kTagMask;
    }
}

__global__ void k_chain_len(const int* __restrict__ cstart, int C, int n, int* __restrict__ clen,
                            int* __restrict__ max_len) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    const int len = (c + 1 < C ? cstart[c + 1] : n) - cstart[c];
    clen[c] = len;
    atomicMax(max_len, len);
}

// ------------------------------------------------------------------ sort

struct BrickGeom {
    int nbx, nby;  // bricks per axis (x, y)
};

__global__ void k_chain_keys(StateBuf st, const int* __restrict__ cstart, int C, MeshGeom g,
                             BrickGeom b, uint32_t* __restrict__ key,
                             uint32_t* __restrict__ count) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    const int i = cstart[c];
    const int cx = axis_coord(st.x[i], g.inv_h[0], g.mx, g.inv_m[0]).lo;
    const int cy = axis_coord(st.y[i], g.inv_h[1], g.my, g.inv_m[1]).lo;
    const int cz = axis_coord(st.z[i], g.inv_h[2], g.mz, g.inv_m[2]).lo;
    const uint32_t brick = (uint32_t)(((cz / kBrick) * b.nby + cy / kBrick) * b.nbx + cx / kBrick);
    const uint32_t in = (uint32_t)(((cz % kBrick) * kBrick + cy % kBrick) * kBrick + cx % kBrick);
    const uint32_t k = brick * (kBrick * kBrick * kBrick) + in;
    key[c] = k;
    atomicAdd(count + k, 1u);
}

__global__ void k_bin_fill(const uint32_t* __restrict__ key, int C,
                           const uint32_t* __restrict__ binoff, uint32_t* __restrict__ cursor,
                           int* __restrict__ order_tmp) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    const uint32_t k = key[c];
    order_tmp[binoff[k] + atomicAdd(cursor + k, 1u)] = c;
}

// Rank each chain inside its bucket by first-bead tag: the final order does
// not depend on the order in which the atomics filled the bucket.
__global__ void k_bin_rank(const int* __restrict__ order_tmp, int C,
                           const uint32_t* __restrict__ key, const uint32_t* __restrict__ binoff,
                           const uint32_t* __restrict__ count, const uint32_t* __restrict__ tag0,
                           const int* __restrict__ clen, int* __restrict__ rank_of,
                           uint32_t* __restrict__ newlen) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= C) return;
    const int c = order_tmp[p];
    const uint32_t k = key[c];
    const uint32_t o = binoff[k], cnt = count[k], t = tag0[c];
    uint32_t r = 0;
    for (uint32_t q = o; q < o + cnt; ++q) r += tag0[order_tmp[q]] < t ? 1u : 0u;
    rank_of[c] = (int)(o + r);
    newlen[o + r] = (uint32_t)clen[c];
}

// Move every bead to its chain's new place (state, meta and chain id).
__global__ void k_permute_beads(StateBuf in, StateBuf out, const uint32_t* __restrict__ meta_in,
                                uint32_t* __restrict__ meta_out,
                                const int* __restrict__ chain_of_in,
                                int* __restrict__ chain_of_out, const int* __restrict__ cstart,
                                const int* __restrict__ rank_of,
                                const uint32_t* __restrict__ newstart, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int c = chain_of_in[i];
    const int j = (int)newstart[rank_of[c]] + (i - cstart[c]);
    out.x[j] = in.x[i];
    out.y[j] = in.y[i];
    out.z[j] = in.z[i];
    out.vx[j] = in.vx[i];
    out.vy[j] = in.vy[i];
    out.vz[j] = in.vz[i];
    meta_out[j] = meta_in[i];
    chain_of_out[j] = c;
}

__global__ void k_update_cstart(const int* __restrict__ rank_of,
                                const uint32_t* __restrict__ newstart, int C,
                                int* __restrict__ cstart) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < C) cstart[c] = (int)newstart[rank_of[c]];
}

// ------------------------------------------------------------------ warp segments
//
// Consecutive whole chains (in storage order) are packed greedily into
// segments of at most kSegBeads beads, one warp per segment.  Each thread
// packs one chunk of kPackChunk chain positions sequentially (segments do not
// straddle chunks), then the per-chunk segment lists are concatenated.
constexpr int kPackChunk = 256;
constexpr int kSegBeads = 64;

__global__ void k_pack_chunks(const uint32_t* __restrict__ newstart, int C, int n,
                              int* __restrict__ tmp_start, int* __restrict__ tmp_count,
                              uint32_t* __restrict__ chunk_nseg) {
    const int chunk = blockIdx.x * blockDim.x + threadIdx.x;
    const int p0 = chunk * kPackChunk;
    if (p0 >= C) return;
    const int p1 = min(C, p0 + kPackChunk);
    int cur_start = 0, cur_count = 0, k = 0;
    for (int p = p0; p < p1; ++p) {
        const int st = (int)newstart[p];
        const int len = (p + 1 < C ? (int)newstart[p + 1] : n) - st;
        if (cur_count > 0 && cur_count + len > kSegBeads) {
            tmp_start[p0 + k] = cur_start;
            tmp_count[p0 + k] = cur_count;
            ++k;
            cur_count = 0;
        }
        if (cur_count == 0) cur_start = st;
        cur_count += len;
    }
    tmp_start[p0 + k] = cur_start;
    tmp_count[p0 + k] = cur_count;
    chunk_nseg[chunk] = (uint32_t)(k + 1);
}

__global__ void k_gather_segments(const int* __restrict__ tmp_start,
                                  const int* __restrict__ tmp_count,
                                  const uint32_t* __restrict__ chunk_nseg,
                                  const uint32_t* __restrict__ chunk_off, int C, int n_chunks,
                                  int* __restrict__ seg_start, int* __restrict__ seg_count,
                                  int* __restrict__ n_seg) {
    const int slot = blockIdx.x * blockDim.x + threadIdx.x;
    if (slot >= C) return;
    const int chunk = slot / kPackChunk, k = slot % kPackChunk;
    if (k < (int)chunk_nseg[chunk]) {
        const int w = (int)chunk_off[chunk] + k;
        seg_start[w] = tmp_start[slot];
        seg_count[w] = tmp_count[slot];
    }
    if (slot == 0) *n_seg = (int)(chunk_off[n_chunks - 1] + chunk_nseg[n_chunks - 1]);
}

// ------------------------------------------------------------------ host side

long long sort_key_space(const MeshGeom& g) {
    const long long nbx = (g.mx + kBrick - 1) / kBrick, nby = (g.my + kBrick - 1) / kBrick,
                    nbz = (g.mz + kBrick - 1) / kBrick;
    return nbx * nby * nbz * kBrick * kBrick * kBrick;
}

int launch_chain_build_heads(const uint32_t* meta, int n, uint32_t* hd, uint32_t* scratch,
                             cudaStream_t s) {
    if (n <= 0) return 0;
    k_heads<<<(n + 255) / 256, 256, 0, s>>>(meta, n, hd);
    return 1 + scan_exclusive(hd, hd, n, scratch, s);  // hd now holds the exclusive scan
}

int launch_chain_build(const uint32_t* meta, const uint32_t* hx, int n, int C, int* cstart,
                       uint32_t* tag0, int* chain_of, int* clen, int* max_len, cudaStream_t s) {
    if (n <= 0) return 0;
    k_chain_build<<<(n + 255) / 256, 256, 0, s>>>(meta, hx, n, cstart, tag0, chain_of);
    k_chain_len<<<(C + 255) / 256, 256, 0, s>>>(cstart, C, n, clen, max_len);
    return 2;
}

int launch_sort(const SortBufs& b, StateBuf in, StateBuf out, const uint32_t* meta_in,
                uint32_t* meta_out, int n, int C, MeshGeom g, cudaStream_t s) {
    if (n <= 0 || C <= 0) return 0;
    const long long K = sort_key_space(g);
    BrickGeom bg{(g.mx + kBrick - 1) / kBrick, (g.my + kBrick - 1) / kBrick};
    const int cb = (C + 255) / 256, nb = (n + 255) / 256;
    int launched = 0;
    cudaMemsetAsync(b.count, 0, sizeof(uint32_t) * K, s);
    cudaMemsetAsync(b.cursor, 0, sizeof(uint32_t) * K, s);
    k_chain_keys<<<cb, 256, 0, s>>>(in, b.cstart, C, g, bg, b.key, b.count);
    ++launched;
    launched += scan_exclusive(b.count, b.binoff, K, b.scratch, s);
    k_bin_fill<<<cb, 256, 0, s>>>(b.key, C, b.binoff, b.cursor, b.order_tmp);
    k_bin_rank<<<cb, 256, 0, s>>>(b.order_tmp, C, b.key, b.binoff, b.count, b.tag0, b.clen,
                                  b.rank_of, b.newstart);
    launched += 2;
    launched += scan_exclusive(b.newstart, b.newstart, C, b.scratch, s);
    k_permute_beads<<<nb, 256, 0, s>>>(in, out, meta_in, meta_out, b.chain_of_in, b.chain_of_out,
                                       b.cstart, b.rank_of, b.newstart, n);
    k_update_cstart<<<cb, 256, 0, s>>>(b.rank_of, b.newstart, C, b.cstart);
    launched += 2;
    if (b.seg_start) {
        const int n_chunks = (C + kPackChunk - 1) / kPackChunk;
        k_pack_chunks<<<(n_chunks + 127) / 128, 128, 0, s>>>(b.newstart, C, n, b.seg_tmp,
                                                            b.seg_tmp + C, b.chunk_nseg);
        launched += 1 + scan_exclusive(b.chunk_nseg, b.chunk_off, n_chunks, b.scratch, s);
        k_gather_segments<<<cb, 256, 0, s>>>(b.seg_tmp, b.seg_tmp + C, b.chunk_nseg, b.chunk_off,
                                             C, n_chunks, b.seg_start, b.seg_count, b.n_seg);
        ++launched;
    }
    return launched;
}

}  // namespace hpf
