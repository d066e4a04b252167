// Tile autotuner for the stencil kernel: times every valid (spt, tx) on
// lattice-owned scratch fields with CUDA events and keeps the fastest.
#include <algorithm>
#include <vector>

#include "dw_api_internal.cuh"

namespace dw {

int tune_tile(dw_lattice *lat, int prec, int op, int nrhs, cudaStream_t st, bool quick) {
  const size_t bytes = field_bytes(lat, prec, nrhs);
  size_t cap_in = lat->stage_bytes, cap_out = lat->stage_bytes;
  int rc = ensure_buffer(&lat->stage_in, &cap_in, bytes);
  if (rc) return rc;
  rc = ensure_buffer(&lat->stage_out, &cap_out, bytes);
  if (rc) return rc;
  lat->stage_bytes = std::min(cap_in, cap_out);
  if (cudaMemsetAsync(lat->stage_in, 0, bytes, st) != cudaSuccess)
    return cuda_fail(cudaGetLastError(), "tune memset");
  std::vector<double> mf(nrhs, 0.01);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  TileConfig best_t = default_tile(lat, prec, op, nrhs);
  const int reps = quick ? 3 : 5;
  // z-blockings: unblocked, the automatic one and twice that (quick: automatic)
  const int za = auto_zblk(lat, prec);
  std::vector<int> zbs{za};
  if (!quick) {
    if (za != 1) zbs.push_back(1);
    if (lat->dims[2] % (2 * za) == 0) zbs.push_back(2 * za);
  }
  for (int variant = 0; variant < kNumVariants; ++variant)
    for (int spt : {1, 2, 3, 4})
      for (int tx : {32, 64, 96, 128, 192, 256})  // 96, 192: planes of 24 x 24 sites
        for (int zblk : zbs)
          for (int sgrp : {1, 2, 3, 4, 6})
          for (int outer = 0; outer < (nrhs > 1 ? 2 : 1); ++outer) {
            TileConfig t{spt, tx, variant, zblk, sgrp, outer};
            if (quick && tx > 128) continue;
            if (!tile_valid(lat, prec, op, t)) continue;
            // warm-up launch doubles as the validity check
            if (run_dslash(lat, prec, op, lat->stage_out, lat->stage_in, mf.data(), nrhs, st, &t)) {
              cudaGetLastError();
              continue;
            }
            std::vector<float> ms;
            for (int r = 0; r < reps; ++r) {
              cudaEventRecord(e0, st);
              run_dslash(lat, prec, op, lat->stage_out, lat->stage_in, mf.data(), nrhs, st, &t);
              cudaEventRecord(e1, st);
              cudaEventSynchronize(e1);
              float m = 0.f;
              cudaEventElapsedTime(&m, e0, e1);
              ms.push_back(m);
            }
            std::sort(ms.begin(), ms.end());
            const float med = ms[ms.size() / 2];
            if (med < best) {
              best = med;
              best_t = t;
            }
          }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  clear_error();
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "tune synchronize");
  lat->tuned[std::make_tuple(prec, op, nrhs)] = best_t;
  return DW_OK;
}

}  // namespace dw
