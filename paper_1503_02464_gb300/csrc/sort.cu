// Periodic on-device counting sort of particle slots by (cell tile, cell in
// tile).  The paper's particles wander between sub-domains one cell per step
// at most (§2, CFL argument); here the "sub-domains" are the push kernel's
// cell tiles, and regrouping the particles by tile every few steps keeps each
// tile's particles contiguous.  Integer-only: the result is exactly defined
// up to the order of particles sharing a cell.
//
//   hist     rank[p] = atomicAdd(&count[key(cell[p])], 1)   (dead slots: -1)
//   tiles    tile_count[t] = sum of the tile's cell counts
//   scan     tile_start = exclusive scan of tile_count; *d_count = total
//   offsets  count[key] <- tile_start[t] + exclusive scan within the tile;
//            the padding slots of each tile run get dst.cell = -1
//   permute  dst.cell[count[key] + rank[p]] = p    (the source of each slot)
//   gather   dst[q] = src[dst.cell[q]]             (every SoA array)
// The move is written as a gather: each destination slot reads its source,
// so the writes of every array are coalesced.  (A scatter that writes each
// particle to its new slot turns into a scatter of partial sectors once the
// particles have drifted for a few steps: 5x slower at 134M particles.)
#include <cuda_runtime.h>

#include "pic_device.cuh"

namespace pic {

namespace {

struct KeyMap {
  int n0, n1;
  int t0, t1, t2;
  int nt0, nt1;
  int tc;  // cells per tile
  __device__ __forceinline__ int key(int c) const {
    const int i = c % n0;
    const int r = c / n0;
    const int j = r % n1;
    const int k = r / n1;
    const int ti = i / t0, tj = j / t1, tk = k / t2;
    const int tile = ti + nt0 * (tj + nt1 * tk);
    return tile * tc + (i - ti * t0) + t0 * ((j - tj * t1) + t1 * (k - tk * t2));
  }
};

__global__ void k_hist(KeyMap km, const int32_t *__restrict__ cell, const int64_t *__restrict__ d_count,
                       int32_t *__restrict__ count, int32_t *__restrict__ rank) {
  const int64_t n = *d_count;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    const int c = cell[p];
    if (c < 0) {
      rank[p] = -1;
      continue;
    }
    const int key = km.key(c);
    // aggregate lanes of the warp that share a key (sorted input: common)
    const unsigned act = __activemask();
    const unsigned peers = __match_any_sync(act, key);
    const int leader = __ffs(peers) - 1;
    const int lane = threadIdx.x & 31;
    const int nbelow = __popc(peers & ((1u << lane) - 1u));
    int base = 0;
    if (lane == leader) base = atomicAdd(&count[key], __popc(peers));
    base = __shfl_sync(peers, base, leader);
    rank[p] = base + nbelow;
  }
}

// one warp per tile
__global__ void k_tile_sum(const int32_t *__restrict__ count, int64_t ntiles, int tc, int64_t *__restrict__ tsum) {
  const int64_t t = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (t >= ntiles) return;
  const int32_t *c = count + t * tc;
  int64_t s = 0;
  for (int i = lane; i < tc; i += 32) s += c[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) tsum[t] = (s + kTilePad - 1) / kTilePad * kTilePad;  // padded run length
}

// single block exclusive scan of ntiles values -> tile_start[0..ntiles]
__global__ void k_scan_tiles(const int64_t *__restrict__ tsum, int64_t ntiles, int64_t *__restrict__ tile_start,
                             int64_t *__restrict__ d_count) {
  __shared__ int64_t sh[1024];
  const int T = blockDim.x;
  const int64_t per = (ntiles + T - 1) / T;
  const int64_t b = threadIdx.x * per;
  const int64_t e = b + per < ntiles ? b + per : ntiles;
  int64_t local = 0;
  for (int64_t i = b; i < e; ++i) local += tsum[i];
  sh[threadIdx.x] = local;
  __syncthreads();
  // Hillis-Steele inclusive scan over the per-thread sums
  for (int o = 1; o < T; o <<= 1) {
    const int64_t v = threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
    __syncthreads();
    sh[threadIdx.x] += v;
    __syncthreads();
  }
  int64_t run = sh[threadIdx.x] - local;
  for (int64_t i = b; i < e; ++i) {
    tile_start[i] = run;
    run += tsum[i];
  }
  if (threadIdx.x == T - 1) {
    tile_start[ntiles] = sh[T - 1];
    *d_count = sh[T - 1];
  }
}

// one warp per tile: count[key] <- absolute start slot of the key; the
// tile's padding slots in the destination are marked dead
__global__ void k_offsets(int32_t *__restrict__ count, int64_t ntiles, int tc, const int64_t *__restrict__ tile_start,
                          int32_t *__restrict__ dst_cell) {
  const int64_t t = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (t >= ntiles) return;
  int32_t *c = count + t * tc;
  int64_t run = tile_start[t];
  for (int base = 0; base < tc; base += 32) {
    const int i = base + lane;
    const int v = i < tc ? c[i] : 0;
    int incl = v;
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (i < tc) c[i] = (int32_t)(run + incl - v);
    run += __shfl_sync(0xffffffffu, incl, 31);
  }
  if (run + lane < tile_start[t + 1]) dst_cell[run + lane] = -1;
}

// Single block: cut every tile's slot run into items of at most `chunk`
// slots.  Exclusive scan of the per-tile item counts, then each thread
// writes the items of its own run of tiles.
__global__ void k_work_items(const int64_t *__restrict__ tile_start, int64_t ntiles, int64_t chunk,
                             int32_t *__restrict__ work_tile, int64_t *__restrict__ work_pb) {
  __shared__ int64_t sh[1024];
  const int T = blockDim.x;
  const int64_t per = (ntiles + T - 1) / T;
  const int64_t b = threadIdx.x * per;
  const int64_t e = b + per < ntiles ? b + per : ntiles;
  int64_t local = 0;
  for (int64_t t = b; t < e; ++t) local += (tile_start[t + 1] - tile_start[t] + chunk - 1) / chunk;
  sh[threadIdx.x] = local;
  __syncthreads();
  for (int o = 1; o < T; o <<= 1) {
    const int64_t v = threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
    __syncthreads();
    sh[threadIdx.x] += v;
    __syncthreads();
  }
  int64_t w = sh[threadIdx.x] - local;
  for (int64_t t = b; t < e; ++t) {
    for (int64_t p = tile_start[t]; p < tile_start[t + 1]; p += chunk, ++w) {
      work_tile[w] = (int32_t)t;
      work_pb[w] = p;
    }
  }
}

__global__ void k_permute(KeyMap km, const int32_t *__restrict__ cell, const int64_t *__restrict__ n_src,
                          const int32_t *__restrict__ count, const int32_t *__restrict__ rank,
                          int32_t *__restrict__ dst_cell, int64_t capacity, Counters *ctr) {
  const int64_t n = *n_src;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    const int r = rank[p];
    if (r < 0) continue;
    const int64_t q = (int64_t)count[km.key(cell[p])] + r;
    if (!PIC_CHECK(q >= 0 && q < capacity, ctr)) continue;
    dst_cell[q] = (int32_t)p;  // slots stay below 2^31
  }
}

template <class R>
__global__ void k_gather(int dims, Particles src, Particles dst, const int64_t *__restrict__ n_dst,
                         const int64_t *__restrict__ n_src, Counters *ctr) {
  const int64_t n = *n_dst;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
    const int p = dst.cell[q];
    if (p < 0) continue;  // tile padding: stays a dead slot
    if (!PIC_CHECK(p < *n_src, ctr)) continue;
    dst.cell[q] = src.cell[p];
    dst.id[q] = src.id[p];
    static_cast<R *>(dst.w)[q] = static_cast<const R *>(src.w)[p];
    for (int d = 0; d < 3; ++d) {
      if (d < dims) static_cast<R *>(dst.off[d])[q] = static_cast<const R *>(src.off[d])[p];
      static_cast<R *>(dst.u[d])[q] = static_cast<const R *>(src.u[d])[p];
    }
  }
}

}  // namespace

cudaError_t launch_sort(const Grid &g, const Particles &src, const Particles &dst, int64_t *d_count,
                        int64_t capacity, int32_t *keys, int32_t *rank, int64_t *tile_start, int64_t *tile_tmp,
                        const WorkSplit &ws, Counters *ctr, cudaStream_t st, int *nlaunch) {
  KeyMap km;
  km.n0 = g.n[0];
  km.n1 = g.n[1];
  km.t0 = g.tile[0];
  km.t1 = g.tile[1];
  km.t2 = g.tile[2];
  km.nt0 = g.ntile[0];
  km.nt1 = g.ntile[1];
  km.tc = g.tile[0] * g.tile[1] * g.tile[2];
  const int64_t nkeys = g.ntiles * km.tc;
  cudaError_t e = cudaMemsetAsync(keys, 0, sizeof(int32_t) * nkeys, st);
  if (e != cudaSuccess) return e;
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int64_t want = (capacity + 255) / 256;
  const int nb = (int)(want < (int64_t)nsm * 16 ? (want > 0 ? want : 1) : (int64_t)nsm * 16);
  // d_count holds the old slot count until the tile scan rewrites it; the
  // scatter reads the old count from tile_tmp[ntiles].
  k_hist<<<nb, 256, 0, st>>>(km, src.cell, d_count, keys, rank);
  const unsigned wb = (unsigned)((g.ntiles * 32 + 255) / 256);
  k_tile_sum<<<wb, 256, 0, st>>>(keys, g.ntiles, km.tc, tile_tmp);
  e = cudaMemcpyAsync(tile_tmp + g.ntiles, d_count, sizeof(int64_t), cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return e;
  k_scan_tiles<<<1, 1024, 0, st>>>(tile_tmp, g.ntiles, tile_start, d_count);
  k_offsets<<<wb, 256, 0, st>>>(keys, g.ntiles, km.tc, tile_start, dst.cell);
  k_permute<<<nb, 256, 0, st>>>(km, src.cell, tile_tmp + g.ntiles, keys, rank, dst.cell, capacity, ctr);
  if (g.prec == 1)
    k_gather<double><<<nb, 256, 0, st>>>(g.dims, src, dst, d_count, tile_tmp + g.ntiles, ctr);
  else
    k_gather<float><<<nb, 256, 0, st>>>(g.dims, src, dst, d_count, tile_tmp + g.ntiles, ctr);
  e = cudaMemsetAsync(ws.work_tile, 0xff, sizeof(int32_t) * (size_t)ws.nwork, st);  // -1: no work
  if (e != cudaSuccess) return e;
  k_work_items<<<1, 1024, 0, st>>>(tile_start, g.ntiles, ws.chunk, ws.work_tile, ws.work_pb);
  if (nlaunch) *nlaunch = 7;
  return cudaGetLastError();
}

}  // namespace pic
