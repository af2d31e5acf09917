// Connected-component labelling of the fragment cells that k_frag_mark has
// marked (a.frag[i] = i on fragment cells, -1 elsewhere).  Fragments are the
// components under face adjacency; periodic faces wrap.
//
// Union-find on the parent array: a link always points a root at a smaller
// root (atomicCAS on the larger one, so two links can never cross), and the
// finds compress paths by writing ancestors.  Every write therefore leaves
// parent[i] <= i with parent[i] in i's component, a walk to the root strictly
// decreases the index, and each component's root ends as its smallest cell
// index: the label is unique and independent of the order of the unions.
#include "mm_internal.h"
#include "mmfrac.h"

namespace {

constexpr int kThreads = 256;
constexpr int kPerThread = MM_FRAG_CELLS / kThreads;  // cells per thread in the ordered count
static_assert(MM_FRAG_CELLS % kThreads == 0, "block of cells must split over the threads");
// A union retries only after another thread linked its root, and each retry
// starts from a strictly smaller root; the cap only turns a broken invariant
// into an error.
constexpr int kUniteRetries = 1 << 22;

int blocks_for(long long n, int threads) {
  long long b = (n + threads - 1) / threads;
  if (b > 152LL * 32) b = 152LL * 32;
  if (b < 1) b = 1;
  return (int)b;
}

__device__ __forceinline__ void frag_report(DevErr* e, int code, long long cell) {
  if (atomicCAS(&e->code, 0, code) == 0) {
    e->cell = cell;
    e->step = 0;
  }
}

// Steps of one walk to a root.  The walk ends by the invariant (indices
// strictly decrease); the cap makes that independent of it: a walk that
// reaches it returns -1 and the caller reports MM_ETIMEOUT.
constexpr int kWalkSteps = 1 << 26;

// Root of i (-1 past the cap).  Loads bypass L1 (ld.global.cg): links made
// by other blocks during the same launch must be seen.  Path halving: each
// visited cell is pointed at its grandparent, an ancestor, which keeps the
// invariant.
__device__ __forceinline__ int find_root(int* parent, int i) {
  int p = __ldcg(parent + i);
  for (int k = 0; p != i; ++k) {
    if (k == kWalkSteps) return -1;
    const int gp = __ldcg(parent + p);
    if (gp != p) parent[i] = gp;
    i = p;
    p = gp;
  }
  return i;
}

// Root of i without writes (-1 past the cap).  The pass that stores every
// cell's root uses it: a halving store from another thread, of an ancestor
// read before the owner stored the root, could otherwise land last and
// leave a non-root.
__device__ __forceinline__ int find_root_ro(const int* parent, int i) {
  int p = __ldcg(parent + i);
  for (int k = 0; p != i; ++k) {
    if (k == kWalkSteps) return -1;
    i = p;
    p = __ldcg(parent + i);
  }
  return i;
}

__device__ __forceinline__ bool unite(int* parent, int a, int b) {
  for (int it = 0; it < kUniteRetries; ++it) {
    a = find_root(parent, a);
    b = find_root(parent, b);
    if (a < 0 || b < 0) return false;
    if (a == b) return true;
    if (a > b) {
      const int t = a;
      a = b;
      b = t;
    }
    if (atomicCAS(parent + b, b, a) == b) return true;
    // b was linked meanwhile: go again from its new root
  }
  return false;
}

struct Geo {
  int n[3];
  int per[3];  // periodic along the axis (both faces)
  int dim;
};

// Joins face neighbours.  Inside a warp's 32 cells the x-runs are linked
// already (k_frag_mark), so an x-union is needed only from a warp's last
// lane to the next cell, and across a periodic x face.  Along y and z, two
// cells i, j = i + stride are joined unless i - 1 and j - 1 are fragment
// cells as well: those two are joined (or skipped for the same reason, down
// to the first cell of the overlap), and i - 1 ~ i, j - 1 ~ j along x, so
// one union per overlap of runs in neighbouring rows covers it.
__global__ void __launch_bounds__(kThreads) k_frag_merge(int* parent, Geo g, long long ncell,
                                                         DevErr* err) {
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  const int sxy = nx * ny;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell;
       c += (long long)gridDim.x * blockDim.x) {
    // membership never changes during the labelling, so a plain load decides it
    if (parent[c] < 0) continue;
    const int i = (int)c;
    const int x = i % nx;
    const int yz = i / nx;
    bool ok = true;
    if (x + 1 < nx) {
      if ((i & 31) == 31 && parent[i + 1] >= 0) ok = unite(parent, i, i + 1);
    } else if (g.per[0] && nx > 1 && parent[i - (nx - 1)] >= 0) {
      ok = unite(parent, i, i - (nx - 1));
    }
    if (g.dim > 1) {
      const int y = yz % ny;
      int j = -1;
      if (y + 1 < ny)
        j = i + nx;
      else if (g.per[1] && ny > 1)
        j = i - (ny - 1) * nx;
      if (j >= 0 && parent[j] >= 0 && !(x > 0 && parent[i - 1] >= 0 && parent[j - 1] >= 0))
        ok = unite(parent, i, j) && ok;
    }
    if (g.dim > 2) {
      const int z = yz / ny;
      int j = -1;
      if (z + 1 < nz)
        j = i + sxy;
      else if (g.per[2] && nz > 1)
        j = i - (nz - 1) * sxy;
      if (j >= 0 && parent[j] >= 0 && !(x > 0 && parent[i - 1] >= 0 && parent[j - 1] >= 0))
        ok = unite(parent, i, j) && ok;
    }
    if (!ok) frag_report(err, MM_ETIMEOUT, c);
  }
}

__global__ void __launch_bounds__(kThreads) k_frag_compress(int* parent, long long ncell,
                                                            DevErr* err) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell;
       c += (long long)gridDim.x * blockDim.x)
    if (parent[c] >= 0) {
      const int r = find_root_ro(parent, (int)c);
      if (r < 0)
        frag_report(err, MM_ETIMEOUT, c);
      else
        parent[c] = r;
    }
}

// Roots in each block of MM_FRAG_CELLS cells (thread t takes cells
// t*kPerThread .. of its block, so that the block's count and the ranks in
// k_frag_ids follow cell order).
__global__ void __launch_bounds__(kThreads) k_frag_block_count(const int* parent, long long ncell,
                                                               int* count) {
  const long long base = (long long)blockIdx.x * MM_FRAG_CELLS + threadIdx.x * kPerThread;
  int k = 0;
  for (int q = 0; q < kPerThread; ++q) {
    const long long c = base + q;
    if (c < ncell && parent[c] == c) ++k;
  }
  for (int o = 16; o > 0; o >>= 1) k += __shfl_xor_sync(0xffffffffu, k, o);
  __shared__ int w[kThreads / 32];
  if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = k;
  __syncthreads();
  if (threadIdx.x == 0) {
    int s = 0;
    for (int i = 0; i < kThreads / 32; ++i) s += w[i];
    count[blockIdx.x] = s;
  }
}

// Exclusive scan of nb block counts in place (one block); boff[nb] = total.
__global__ void __launch_bounds__(1024) k_frag_scan(int* boff, int nb) {
  __shared__ int part[1024];
  const int per = (nb + 1023) / 1024;
  const int lo = threadIdx.x * per;
  int s = 0;
  for (int i = lo; i < lo + per && i < nb; ++i) s += boff[i];
  part[threadIdx.x] = s;
  __syncthreads();
  // Hillis-Steele inclusive scan of the 1024 partial sums
  for (int o = 1; o < 1024; o <<= 1) {
    const int v = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  int run = threadIdx.x == 0 ? 0 : part[threadIdx.x - 1];
  for (int i = lo; i < lo + per && i < nb; ++i) {
    const int v = boff[i];
    boff[i] = run;
    run += v;
  }
  if (threadIdx.x == 1023) boff[nb] = part[1023];
}

// Fragment number of every root, in cell order: the block's offset plus the
// roots before it in the block.
__global__ void __launch_bounds__(kThreads) k_frag_ids(const int* parent, long long ncell,
                                                       const int* boff, int* fid,
                                                       long long* flabel) {
  const long long base = (long long)blockIdx.x * MM_FRAG_CELLS + threadIdx.x * kPerThread;
  int k = 0;
  for (int q = 0; q < kPerThread; ++q) {
    const long long c = base + q;
    if (c < ncell && parent[c] == c) ++k;
  }
  // exclusive scan of k over the block
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int inc = k;
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += v;
  }
  __shared__ int w[kThreads / 32];
  if (lane == 31) w[wid] = inc;
  __syncthreads();
  int before = 0;
  for (int i = 0; i < wid; ++i) before += w[i];
  int r = boff[blockIdx.x] + before + inc - k;
  for (int q = 0; q < kPerThread; ++q) {
    const long long c = base + q;
    if (c < ncell && parent[c] == c) {
      fid[c] = r;
      flabel[r] = c;
      ++r;
    }
  }
}

// Per-fragment sums.  Neighbouring cells nearly always share a fragment:
// warps without fragment cells skip, the other lanes of a warp join its
// first fragment cell's fragment with nothing to add, and a warp whose
// cells then all name one fragment adds its count and mass with one atomic
// each; only warps that span two fragments combine lane by lane.  Whole
// warps run the loop (bound rounded up to the warp) so that every shuffle
// has all 32 lanes.
__global__ void __launch_bounds__(kThreads) k_frag_accum(const int* parent, const double* cm,
                                                         long long ncell, const int* fid,
                                                         unsigned long long* fcells,
                                                         double* fmass) {
  const unsigned full = 0xffffffffu;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long end = (ncell + 31) / 32 * 32;
  const int lane = threadIdx.x & 31;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < end; c += stride) {
    const int r = c < ncell ? parent[c] : -1;
    const unsigned mem = __ballot_sync(full, r >= 0);
    if (mem == 0) continue;
    const int lead = __ffs(mem) - 1;
    const int f = r >= 0 ? fid[r] : -1;
    const int f0 = __shfl_sync(full, f, lead);
    const int fe = r >= 0 ? f : f0;
    double m = r >= 0 ? cm[c] : 0.0;
    if (__ballot_sync(full, fe == f0) == full) {
      for (int o = 16; o > 0; o >>= 1) m += __shfl_xor_sync(full, m, o);
      if (lane == lead) {
        atomicAdd(fcells + f0, (unsigned long long)__popc(mem));
        atomicAdd(fmass + f0, m);
      }
    } else {
      double sm = 0.0;
      unsigned k = 0;
      int first = 32;
      for (int src = 0; src < 32; ++src) {
        const int fs = __shfl_sync(full, fe, src);
        const double ms = __shfl_sync(full, m, src);
        if (fs == fe) {
          sm += ms;
          k += (mem >> src) & 1u;
          if (first == 32) first = src;
        }
      }
      if (first == lane) {
        atomicAdd(fcells + fe, (unsigned long long)k);
        atomicAdd(fmass + fe, sm);
      }
    }
  }
}

}  // namespace

cudaError_t mm_frag_label(const KArgs& a, cudaStream_t s) {
  Geo g;
  g.dim = a.dim;
  for (int d = 0; d < 3; ++d) {
    g.n[d] = d < a.dim ? a.n[d] : 1;
    g.per[d] = d < a.dim && a.bc[d][0] == MM_BC_PERIODIC && a.bc[d][1] == MM_BC_PERIODIC;
  }
  const int nb = blocks_for(a.ncell, kThreads);
  k_frag_merge<<<nb, kThreads, 0, s>>>(a.frag, g, a.ncell, a.err);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_frag_compress<<<nb, kThreads, 0, s>>>(a.frag, a.ncell, a.err);
  return cudaGetLastError();
}

cudaError_t mm_frag_count(const KArgs& a, int* boff, cudaStream_t s) {
  const long long nblk = (a.ncell + MM_FRAG_CELLS - 1) / MM_FRAG_CELLS;
  k_frag_block_count<<<(unsigned)nblk, kThreads, 0, s>>>(a.frag, a.ncell, boff);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_frag_scan<<<1, 1024, 0, s>>>(boff, (int)nblk);
  return cudaGetLastError();
}

cudaError_t mm_frag_collect(const KArgs& a, const int* boff, int* fid, long long* flabel,
                            unsigned long long* fcells, double* fmass, cudaStream_t s) {
  const long long nblk = (a.ncell + MM_FRAG_CELLS - 1) / MM_FRAG_CELLS;
  k_frag_ids<<<(unsigned)nblk, kThreads, 0, s>>>(a.frag, a.ncell, boff, fid, flabel);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_frag_accum<<<blocks_for(a.ncell, kThreads), kThreads, 0, s>>>(a.frag, a.fmass, a.ncell, fid,
                                                                   fcells, fmass);
  return cudaGetLastError();
}
