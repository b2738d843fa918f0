// Mesh registration: triangle adjacency across shared undirected edges {a, b},
// a != b (the half-edge twins that Alg. 1 walks), built once per mesh on the
// device with an open-addressing hash table of edge keys.
//   adj[3t + j] = the other triangle on edge (v_j, v_{j+1}) when exactly two
//                 triangle edges carry that key, -1 when one does, and -2 - e for
//                 non-manifold edge e (three or more), whose incident triangles are
//                 listed in nm_list[nm_off[e] .. nm_off[e+1]).
#include <vector>

#include "fa_internal.cuh"

namespace fa {
namespace {

constexpr unsigned long long kEmpty = ~0ull;

__device__ __forceinline__ uint32_t hash_key(unsigned long long k) {
  k ^= k >> 33;
  k *= 0xff51afd7ed558ccdull;
  k ^= k >> 33;
  k *= 0xc4ceb9fe1a85ec53ull;
  k ^= k >> 33;
  return (uint32_t)k;
}

struct Table {
  unsigned long long* keys;
  uint32_t* cnt;
  uint32_t* fill;
  int32_t* tri;  // [2 * cap]
  int32_t* slot;  // [3T] slot of each triangle edge, -1 for a == b
  uint32_t* nm_id;  // [cap]
  uint32_t mask;
};

__global__ void k_init_table(Table tb, uint32_t cap) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < cap; i += gridDim.x * blockDim.x) {
    tb.keys[i] = kEmpty;
    tb.cnt[i] = 0;
    tb.fill[i] = 0;
    tb.nm_id[i] = 0xFFFFFFFFu;
  }
}

__global__ void k_insert(Table tb, const uint32_t* idx, uint32_t T, uint32_t V, uint32_t* bad) {
  for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < 3 * T; e += gridDim.x * blockDim.x) {
    const uint32_t t = e / 3, j = e % 3;
    const uint32_t a = idx[3 * (size_t)t + j], b = idx[3 * (size_t)t + (j + 1) % 3];
    if (a >= V || b >= V) {
      atomicAdd(bad, 1u);
      tb.slot[e] = -1;
      continue;
    }
    if (a == b) {
      tb.slot[e] = -1;
      continue;
    }
    const unsigned long long key = ((unsigned long long)min(a, b) << 32) | max(a, b);
    uint32_t h = hash_key(key) & tb.mask;
    for (uint32_t probe = 0; probe <= tb.mask; ++probe) {
      unsigned long long old = atomicCAS(tb.keys + h, kEmpty, key);
      if (old == kEmpty || old == key) break;
      h = (h + 1) & tb.mask;
    }
    tb.slot[e] = (int32_t)h;
    atomicAdd(tb.cnt + h, 1u);
  }
}

__global__ void k_pairs(Table tb, uint32_t T) {
  for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < 3 * T; e += gridDim.x * blockDim.x) {
    const int32_t h = tb.slot[e];
    if (h < 0 || tb.cnt[h] != 2) continue;
    const uint32_t p = atomicAdd(tb.fill + h, 1u);
    tb.tri[2 * h + p] = (int32_t)(e / 3);
  }
}

// Number the non-manifold edges and reserve their incidence ranges.
__global__ void k_nm_number(Table tb, uint32_t cap, uint32_t* n_nm, uint32_t* nm_total,
                            uint32_t* nm_start, uint32_t* nm_cnt, uint32_t max_nm) {
  for (uint32_t h = blockIdx.x * blockDim.x + threadIdx.x; h < cap; h += gridDim.x * blockDim.x) {
    if (tb.keys[h] == kEmpty || tb.cnt[h] < 3) continue;
    const uint32_t id = atomicAdd(n_nm, 1u);
    if (id >= max_nm) continue;
    tb.nm_id[h] = id;
    nm_start[id] = atomicAdd(nm_total, tb.cnt[h]);
    nm_cnt[id] = tb.cnt[h];
  }
}

__global__ void k_adj(Table tb, uint32_t T, int32_t* adj, const uint32_t* nm_start, uint32_t* nm_fill,
                      uint32_t* nm_list) {
  for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < 3 * T; e += gridDim.x * blockDim.x) {
    const int32_t h = tb.slot[e];
    int32_t out = -1;
    if (h >= 0) {
      const uint32_t c = tb.cnt[h];
      const int32_t t = (int32_t)(e / 3);
      if (c == 2) {
        const int32_t a = tb.tri[2 * h], b = tb.tri[2 * h + 1];
        out = (a == t) ? b : a;
      } else if (c >= 3) {
        const uint32_t id = tb.nm_id[h];
        if (id != 0xFFFFFFFFu) {
          const uint32_t p = atomicAdd(nm_fill + id, 1u);
          nm_list[nm_start[id] + p] = (uint32_t)t;
          out = -2 - (int32_t)id;
        }
      }
    }
    adj[e] = out;
  }
}

}  // namespace

fa_status build_adjacency(fa_ctx* ctx, fa_mesh* mesh, cudaStream_t s) {
  const uint32_t T = mesh->T;
  uint32_t cap = 1024;
  while (cap < 3u * T) cap <<= 1;
  if (T == 0) {
    mesh->adj = nullptr;
    mesh->n_nm = 0;
    return FA_OK;
  }
  Table tb;
  tb.mask = cap - 1;
  void* buf = nullptr;
  const size_t bytes = (size_t)cap * (8 + 4 + 4 + 8 + 4) + (size_t)3 * T * 4 + 64;
  if (cudaMalloc(&buf, bytes) != cudaSuccess) return FA_E_OUT_OF_MEMORY;
  char* p = (char*)buf;
  tb.keys = (unsigned long long*)p; p += (size_t)cap * 8;
  tb.tri = (int32_t*)p; p += (size_t)cap * 8;
  tb.cnt = (uint32_t*)p; p += (size_t)cap * 4;
  tb.fill = (uint32_t*)p; p += (size_t)cap * 4;
  tb.nm_id = (uint32_t*)p; p += (size_t)cap * 4;
  tb.slot = (int32_t*)p; p += (size_t)3 * T * 4;
  uint32_t* small = (uint32_t*)p;  // [0] bad, [1] n_nm, [2] nm_total
  fa_status st = FA_OK;
  if (cudaMalloc(&mesh->adj, (size_t)3 * T * 4) != cudaSuccess) {
    cudaFree(buf);
    return FA_E_OUT_OF_MEMORY;
  }
  const unsigned g = grid_for((uint64_t)3 * T, 256, 152 * 16);
  cudaMemsetAsync(small, 0, 16, s);
  k_init_table<<<grid_for(cap, 256, 152 * 16), 256, 0, s>>>(tb, cap);
  k_insert<<<g, 256, 0, s>>>(tb, mesh->idx, T, mesh->V, small);
  k_pairs<<<g, 256, 0, s>>>(tb, T);
  // count non-manifold edges first (sizes the incidence lists)
  uint32_t* d_nm_start = nullptr;
  uint32_t* d_nm_cnt = nullptr;
  const uint32_t max_nm = T;  // an edge key with >= 3 uses needs >= 3 triangle edges
  if (cudaMalloc(&d_nm_start, (size_t)(max_nm + 1) * 4) != cudaSuccess ||
      cudaMalloc(&d_nm_cnt, (size_t)(max_nm + 1) * 4) != cudaSuccess) {
    cudaFree(buf);
    cudaFree(d_nm_start);
    cudaFree(mesh->adj);
    mesh->adj = nullptr;
    return FA_E_OUT_OF_MEMORY;
  }
  k_nm_number<<<grid_for(cap, 256, 152 * 16), 256, 0, s>>>(tb, cap, small + 1, small + 2, d_nm_start,
                                                           d_nm_cnt, max_nm);
  uint32_t host_small[3] = {0, 0, 0};
  if (cudaMemcpyAsync(host_small, small, 12, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    st = FA_E_CUDA;
  }
  ctx->launches += 4;
  if (st == FA_OK && host_small[0] != 0) st = FA_E_INVALID_ARG;  // index out of range
  const uint32_t n_nm = host_small[1], nm_total = host_small[2];
  uint32_t* nm_fill = nullptr;
  mesh->n_nm = 0;
  mesh->nm_off = nullptr;
  mesh->nm_list = nullptr;
  if (st == FA_OK) {
    if (cudaMalloc(&mesh->nm_list, (size_t)(nm_total + 1) * 4) != cudaSuccess ||
        cudaMalloc(&mesh->nm_off, (size_t)(n_nm + 1) * 4) != cudaSuccess ||
        cudaMalloc(&nm_fill, (size_t)(n_nm + 1) * 4) != cudaSuccess) {
      st = FA_E_OUT_OF_MEMORY;
    }
  }
  if (st == FA_OK) {
    cudaMemsetAsync(nm_fill, 0, (size_t)(n_nm + 1) * 4, s);
    k_adj<<<g, 256, 0, s>>>(tb, T, mesh->adj, d_nm_start, nm_fill, mesh->nm_list);
    ctx->launches++;
    // nm_off: the reserved ranges are disjoint but in arbitrary order; keep the
    // start of each edge and its end (start + count) as [start, end) pairs on the host.
    std::vector<uint32_t> hs(n_nm + 1), hc(n_nm + 1);
    if (n_nm) {
      if (cudaMemcpyAsync(hs.data(), d_nm_start, (size_t)n_nm * 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
          cudaMemcpyAsync(hc.data(), d_nm_cnt, (size_t)n_nm * 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
          cudaStreamSynchronize(s) != cudaSuccess) {
        st = FA_E_CUDA;
      }
    }
    if (st == FA_OK && n_nm) {
      // rewrite nm_list so that edge e's triangles are contiguous in id order
      std::vector<uint32_t> list(nm_total);
      if (cudaMemcpy(list.data(), mesh->nm_list, (size_t)nm_total * 4, cudaMemcpyDeviceToHost) != cudaSuccess) {
        st = FA_E_CUDA;
      } else {
        std::vector<uint32_t> out(nm_total), off(n_nm + 1);
        uint32_t o = 0;
        for (uint32_t e = 0; e < n_nm; ++e) {
          off[e] = o;
          for (uint32_t i = 0; i < hc[e]; ++i) out[o++] = list[hs[e] + i];
        }
        off[n_nm] = o;
        if (cudaMemcpy(mesh->nm_list, out.data(), (size_t)nm_total * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(mesh->nm_off, off.data(), (size_t)(n_nm + 1) * 4, cudaMemcpyHostToDevice) != cudaSuccess)
          st = FA_E_CUDA;
      }
    }
    mesh->n_nm = n_nm;
  }
  if (cudaStreamSynchronize(s) != cudaSuccess && st == FA_OK) st = FA_E_CUDA;
  cudaFree(nm_fill);
  cudaFree(d_nm_start);
  cudaFree(d_nm_cnt);
  cudaFree(buf);
  if (st != FA_OK) {
    cudaFree(mesh->adj);
    cudaFree(mesh->nm_list);
    cudaFree(mesh->nm_off);
    mesh->adj = nullptr;
    mesh->nm_list = nullptr;
    mesh->nm_off = nullptr;
    mesh->n_nm = 0;
  }
  return st;
}

}  // namespace fa
