// k_count.cu — the algorithmic cell-face test count of a level (a measurement,
// not part of the refinement): per cell of the level's blocks, the distinct
// faces stored in the bins that the cell's inflated box overlaps.  That is the
// number of tests a cell-by-cell search over the bins would run (Sec. "Spatial
// Binning Algorithm": each cell checks the faces of the bins around it), fixed
// by the geometry and the bin density, whatever the kernels actually execute.
//
// The cell centre, the inflated box and its bin range are formed in FP64 with
// one rounding per operation in the order of the definition, so the count is
// exact.  A face met in several of the box's bins is counted in one of them:
// the first bin of its own range inside the box (the first-bin flags of the
// bin entries, as in the block walk).
#include "internal.cuh"

namespace amr {

namespace {

constexpr int kCThreads = 256;

template <int D>
__global__ void __launch_bounds__(kCThreads) k_count_candidates(CountArgs a) {
  using E = typename EntryT<D>::type;
  constexpr int NC = D == 3 ? 64 : 16;
  const int64_t n = a.n;
  const E* payload = static_cast<const E*>(a.payload);
  unsigned long long count = 0;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n * NC; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t blk = t / NC;
    const int cell = (int)(t % NC);
    const GeomParams& P = a.g0;
    const double h = scalbn(P.h0, -a.level);
    const double dL = __dadd_rn(P.d_abs, __dmul_rn(P.d_rel, h));
    const double r = __dadd_rn(__dmul_rn(0.5, h), dL);
    int qlo[3] = {0, 0, 0}, qhi[3] = {0, 0, 0};
#pragma unroll
    for (int c = 0; c < D; ++c) {
      const int ci = 4 * a.blocks[blk * D + c] + ((cell >> (2 * c)) & 3);
      const double x = __dadd_rn(P.origin[c], __dmul_rn((double)ci + 0.5, h));
      qlo[c] = bin_coord(__dsub_rn(x, r), P.origin[c], P.bin_scale[c], P.B);
      qhi[c] = bin_coord(__dadd_rn(x, r), P.origin[c], P.bin_scale[c], P.B);
    }
    const int64_t B = P.B;
    for (int z = qlo[2]; z <= qhi[2]; ++z)
      for (int y = qlo[1]; y <= qhi[1]; ++y)
        for (int x = qlo[0]; x <= qhi[0]; ++x) {
          const int64_t b = P.bin_base + x + B * (y + B * (int64_t)z);
          const uint32_t e0 = a.offsets[b], e1 = a.offsets[b + 1];
          for (uint32_t e = e0; e < e1; ++e) {
            const uint32_t id = payload[e].id;
            // counted in the face's first bin inside the box: its own first bin, or the box's edge
            bool first = ((id >> 29) & 1u) || x == qlo[0];
            first = first && (((id >> 30) & 1u) || y == qlo[1]);
            if (D == 3) first = first && (((id >> 31) & 1u) || z == qlo[2]);
            count += first ? 1ull : 0ull;
          }
        }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) count += __shfl_xor_sync(0xffffffffu, count, o);
  if ((threadIdx.x & 31) == 0 && count) atomicAdd(a.out, count);
}

}  // namespace

int launch_count_candidates(const CountArgs& a, int num_sms, cudaStream_t st) {
  const int NC = a.dim == 3 ? 64 : 16;
  int64_t g = (a.n * NC + kCThreads - 1) / kCThreads;
  if (g > (int64_t)num_sms * 16) g = (int64_t)num_sms * 16;
  if (g < 1) g = 1;
  if (a.dim == 3)
    k_count_candidates<3><<<(unsigned)g, kCThreads, 0, st>>>(a);
  else
    k_count_candidates<2><<<(unsigned)g, kCThreads, 0, st>>>(a);
  return 1;
}

}  // namespace amr
