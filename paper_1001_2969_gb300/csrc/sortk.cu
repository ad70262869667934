// sortk.cu -- the per-step cell sort of the particle store and the canonical
// numbering of newborn particles.
//
// Cell sort: counts per cell (made by the particle pass), an exclusive scan
// into per-cell cursors, then a rank pass that writes the permutation the
// next pass reads through.  Dead particles (cell -1) are left out, so the
// sort also compacts.  Order inside a cell is not fixed.
//
// Newborns are numbered next_id + rank of their key (parent species, parent
// id, birth slot): one block ranks small batches directly, larger batches
// go through an LSD radix sort of (key, index) pairs.
#include "pic_internal.cuh"

namespace pic {

template <typename T>
__global__ void k_hist(PBuf<T> buf, const int32_t *n_dev, int32_t *counts) {
    const int n = *n_dev;
    const int lane = threadIdx.x & 31;
    for (int base = blockIdx.x * blockDim.x; base < n; base += gridDim.x * blockDim.x) {
        const int k = base + threadIdx.x;
        const int c = k < n ? buf.cell[k] : -1;
        const unsigned peers = __match_any_sync(0xffffffffu, c);
        if (c >= 0 && lane == __ffs(peers) - 1) atomicAdd(counts + c, __popc(peers));
    }
}

template <typename T>
void launch_hist(PBuf<T> buf, const int32_t *n_dev, int32_t *counts, cudaStream_t st) {
    k_hist<T><<<152 * 8, 256, 0, st>>>(buf, n_dev, counts);
}

// ---- exclusive scan over cells: tiles of 4096 (1024 threads x 4) ----
constexpr int kScanThreads = 1024;
constexpr int kScanTile = 4096;

__device__ __forceinline__ int block_exclusive_scan(int v, int *s_warp, int *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int w = lane < (int)(blockDim.x >> 5) ? s_warp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        s_warp[lane] = w;  // inclusive over warps
    }
    __syncthreads();
    const int warp_excl = warp > 0 ? s_warp[warp - 1] : 0;
    if (total) *total = s_warp[(blockDim.x >> 5) - 1];
    return warp_excl + x - v;
}

__global__ void k_scan_tiles(const int32_t *counts, int ncell, int32_t *block_sums) {
    __shared__ int s_warp[32];
    const int base = blockIdx.x * kScanTile + threadIdx.x * 4;
    int v = 0;
    for (int q = 0; q < 4; ++q) v += (base + q < ncell) ? counts[base + q] : 0;
    int tot;
    block_exclusive_scan(v, s_warp, &tot);
    if (threadIdx.x == 0) block_sums[blockIdx.x] = tot;
}

__global__ void k_scan_top(int32_t *block_sums, int nblocks, int32_t *n_alive, int64_t capacity,
                           DevScalars *ds) {
    __shared__ int s_warp[32];
    __shared__ int s_carry;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (int b0 = 0; b0 < nblocks; b0 += blockDim.x) {
        const int k = b0 + threadIdx.x;
        const int v = k < nblocks ? block_sums[k] : 0;
        int tot;
        const int ex = block_exclusive_scan(v, s_warp, &tot);
        const int carry = s_carry;
        if (k < nblocks) block_sums[k] = carry + ex;
        __syncthreads();
        if (threadIdx.x == 0) s_carry = carry + tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        *n_alive = s_carry;
        if ((int64_t)s_carry > capacity) atomicOr(&ds->status, ST_CAPACITY);
    }
}

__global__ void k_scan_apply(const int32_t *counts, int ncell, const int32_t *block_sums,
                             int32_t *cursor) {
    __shared__ int s_warp[32];
    const int base = blockIdx.x * kScanTile + threadIdx.x * 4;
    int c[4];
    int v = 0;
    for (int q = 0; q < 4; ++q) {
        c[q] = (base + q < ncell) ? counts[base + q] : 0;
        v += c[q];
    }
    int ex = block_exclusive_scan(v, s_warp, nullptr) + block_sums[blockIdx.x];
    for (int q = 0; q < 4; ++q) {
        if (base + q < ncell) cursor[base + q] = ex;
        ex += c[q];
    }
}

void launch_scan(const int32_t *counts, int32_t *cursor, int ncell, int32_t *block_sums,
                 int32_t *n_alive, int64_t capacity, DevScalars *ds, cudaStream_t st) {
    const int nb = (ncell + kScanTile - 1) / kScanTile;
    k_scan_tiles<<<nb, kScanThreads, 0, st>>>(counts, ncell, block_sums);
    k_scan_top<<<1, kScanThreads, 0, st>>>(block_sums, nb, n_alive, capacity, ds);
    k_scan_apply<<<nb, kScanThreads, 0, st>>>(counts, ncell, block_sums, cursor);
}

// ---- rank: perm[cursor[cell]++] = element (main first, then births) ----
template <typename T>
__global__ void k_rank(PBuf<T> mainb, const int32_t *n_main_dev, PBuf<T> births,
                       const int32_t *n_births_dev, int32_t *cursor, int32_t *perm,
                       const int32_t *n_alive, int64_t cap, const int32_t *status) {
    // a failed step keeps the previous permutation
    if ((int64_t)*n_alive > cap || (*status & (ST_CAPACITY | ST_BIRTH_OVERFLOW))) return;
    const int nm = *n_main_dev, nb = *n_births_dev;
    const int total = nm + nb;
    const int lane = threadIdx.x & 31;
    for (int base = blockIdx.x * blockDim.x; base < total; base += gridDim.x * blockDim.x) {
        const int e = base + threadIdx.x;
        int c = -1;
        if (e < nm)
            c = mainb.cell[e];
        else if (e < total)
            c = births.cell[e - nm];
        const unsigned peers = __match_any_sync(0xffffffffu, c);
        const int leader = __ffs(peers) - 1;
        int pos = 0;
        if (c >= 0 && lane == leader) pos = atomicAdd(cursor + c, __popc(peers));
        pos = __shfl_sync(peers, pos, leader);
        if (c >= 0) perm[pos + __popc(peers & ((1u << lane) - 1u))] = e;
    }
}

template <typename T>
void launch_rank(PBuf<T> mainb, const int32_t *n_main, PBuf<T> births, const int32_t *n_births,
                 int32_t *cursor, int32_t *perm, const int32_t *n_alive, int64_t cap,
                 const int32_t *status, cudaStream_t st) {
    k_rank<T><<<152 * 8, 256, 0, st>>>(mainb, n_main, births, n_births, cursor, perm, n_alive, cap,
                                        status);
}

// ---- newborn numbering, small batches: rank by counting smaller keys ----
constexpr int kSmallBirths = 2048;

__global__ void k_birth_ids_small(const uint64_t *key, uint64_t *id, int nb, uint64_t next_id) {
    __shared__ uint64_t s_key[kSmallBirths];
    for (int k = threadIdx.x; k < nb; k += blockDim.x) s_key[k] = key[k];
    __syncthreads();
    for (int k = threadIdx.x; k < nb; k += blockDim.x) {
        const uint64_t mine = s_key[k];
        int rank = 0;
        for (int q = 0; q < nb; ++q) rank += s_key[q] < mine;
        id[k] = next_id + (uint64_t)rank;
    }
}

void launch_birth_ids_small(const uint64_t *key, uint64_t *id, int nb, uint64_t next_id,
                            cudaStream_t st) {
    if (nb <= 0) return;
    k_birth_ids_small<<<1, 1024, 0, st>>>(key, id, nb, next_id);
}

// ---- newborn numbering, large batches: LSD radix sort, 8-bit digits ----
constexpr int kRadixThreads = 256;
constexpr int kRadixPer = 8;
constexpr int kRadixTile = kRadixThreads * kRadixPer;

__global__ void k_radix_init(const uint64_t *key, uint64_t *k0, uint32_t *v0, int n) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) {
        k0[e] = key[e];
        v0[e] = (uint32_t)e;
    }
}

__global__ void k_radix_hist(const uint64_t *keys, int n, int shift, uint32_t *hist, int ntiles) {
    __shared__ uint32_t s_h[256];
    s_h[threadIdx.x] = 0;
    __syncthreads();
    const int base = blockIdx.x * kRadixTile;
    for (int q = 0; q < kRadixPer; ++q) {
        const int e = base + q * kRadixThreads + threadIdx.x;
        if (e < n) atomicAdd(&s_h[(keys[e] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[threadIdx.x * ntiles + blockIdx.x] = s_h[threadIdx.x];
}

__global__ void k_radix_scan(uint32_t *hist, int total) {
    __shared__ int s_warp[32];
    __shared__ int s_carry;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (int b0 = 0; b0 < total; b0 += blockDim.x) {
        const int k = b0 + threadIdx.x;
        const int v = k < total ? (int)hist[k] : 0;
        int tot;
        const int ex = block_exclusive_scan(v, s_warp, &tot);
        const int carry = s_carry;
        if (k < total) hist[k] = (uint32_t)(carry + ex);
        __syncthreads();
        if (threadIdx.x == 0) s_carry = carry + tot;
        __syncthreads();
    }
}

// stable scatter of one tile: rounds of 256 keys in order; inside a round a
// key's place is (keys of its digit in earlier warps) + (earlier lanes of
// its warp with the same digit)
__global__ void k_radix_scatter(const uint64_t *kin, const uint32_t *vin, uint64_t *kout,
                                uint32_t *vout, int n, int shift, const uint32_t *hist,
                                int ntiles) {
    __shared__ uint32_t s_run[256];
    __shared__ uint32_t s_wc[kRadixThreads / 32][256];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    s_run[tid] = hist[tid * ntiles + blockIdx.x];
    for (int w = 0; w < kRadixThreads / 32; ++w) s_wc[w][tid] = 0;
    __syncthreads();
    const int base = blockIdx.x * kRadixTile;
    for (int q = 0; q < kRadixPer; ++q) {
        const int e = base + q * kRadixThreads + tid;
        const bool valid = e < n;
        uint64_t key = valid ? kin[e] : 0;
        const int d = valid ? (int)((key >> shift) & 255u) : 256 + lane;  // unique dummies
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int rank_w = __popc(peers & ((1u << lane) - 1u));
        if (valid && lane == __ffs(peers) - 1) s_wc[warp][d] = __popc(peers);
        __syncthreads();
        if (valid) {
            uint32_t off = s_run[d];
            for (int w = 0; w < warp; ++w) off += s_wc[w][d];
            const uint32_t pos = off + (uint32_t)rank_w;
            kout[pos] = key;
            vout[pos] = vin[e];
        }
        __syncthreads();
        uint32_t add = 0;
        for (int w = 0; w < kRadixThreads / 32; ++w) {
            add += s_wc[w][tid];
            s_wc[w][tid] = 0;
        }
        s_run[tid] += add;
        __syncthreads();
    }
}

__global__ void k_radix_ids(const uint32_t *v, uint64_t *id, int n, uint64_t next_id) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n) id[v[r]] = next_id + (uint64_t)r;
}

void launch_birth_ids_radix(const uint64_t *key, uint64_t *id, int nb, uint64_t next_id,
                            RadixTmp t, int *launches, cudaStream_t st) {
    if (nb <= 0) return;
    const int ntiles = (nb + kRadixTile - 1) / kRadixTile;
    k_radix_init<<<(nb + 255) / 256, 256, 0, st>>>(key, t.k0, t.v0, nb);
    int L = 1;
    uint64_t *ka = t.k0, *kb = t.k1;
    uint32_t *va = t.v0, *vb = t.v1;
    for (int shift = 0; shift < 64; shift += 8) {
        k_radix_hist<<<ntiles, kRadixThreads, 0, st>>>(ka, nb, shift, t.hist, ntiles);
        k_radix_scan<<<1, 1024, 0, st>>>(t.hist, 256 * ntiles);
        k_radix_scatter<<<ntiles, kRadixThreads, 0, st>>>(ka, va, kb, vb, nb, shift, t.hist, ntiles);
        L += 3;
        uint64_t *tk = ka;
        ka = kb;
        kb = tk;
        uint32_t *tv = va;
        va = vb;
        vb = tv;
    }
    k_radix_ids<<<(nb + 255) / 256, 256, 0, st>>>(va, id, nb, next_id);
    L += 1;
    if (launches) *launches += L;
}

template void launch_hist<float>(PBuf<float>, const int32_t *, int32_t *, cudaStream_t);
template void launch_hist<double>(PBuf<double>, const int32_t *, int32_t *, cudaStream_t);
template void launch_rank<float>(PBuf<float>, const int32_t *, PBuf<float>, const int32_t *,
                                 int32_t *, int32_t *, const int32_t *, int64_t, const int32_t *,
                                 cudaStream_t);
template void launch_rank<double>(PBuf<double>, const int32_t *, PBuf<double>, const int32_t *,
                                  int32_t *, int32_t *, const int32_t *, int64_t, const int32_t *,
                                  cudaStream_t);

}  // namespace pic
