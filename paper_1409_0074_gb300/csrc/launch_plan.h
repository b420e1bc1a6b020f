// launch_plan.h -- host-side launch arithmetic of the persistent and tiled
// kernels, kept free of CUDA so that it compiles and is tested on any host.
#pragma once
#include <cstddef>
#include <cstdint>

namespace lagp {

// The tensor-core kNN filter runs one CTA per SM (it takes all 512 TMEM
// columns) over `tiles` location tiles, each streaming `design_tiles` design
// tiles.  Tiles [0, *body) run unsplit in whole waves; the remaining
// tiles - *body run with the design split into *nseg segments (one CTA
// each).  A batch with fewer tiles than SMs splits every tile, about two CTAs
// per SM; a larger batch splits the tiles of its last, partial wave over the
// SMs that wave would leave idle.  A segment keeps at least 64 design tiles.
inline void knn_tc_plan(int64_t tiles, int64_t sms, int64_t design_tiles, int64_t* body,
                        int64_t* nseg) {
  int64_t b = tiles, s = 1;
  if (tiles > 0 && tiles < sms) {
    s = (2 * sms + tiles - 1) / tiles;
    b = 0;
  } else if (sms > 0 && tiles % sms != 0) {
    s = sms / (tiles % sms);
    b = tiles - tiles % sms;
  }
  if (s > design_tiles / 64) s = design_tiles / 64;
  if (s > 65535) s = 65535;
  if (s < 2) { s = 1; b = tiles; }
  *body = b;
  *nseg = s;
}

// Warps per CTA (2, 4 or 1) of a kernel whose warps each take `warp_bytes` of
// shared memory, so that the most warps reside on an SM with `smem_sm` bytes
// and `reserved` bytes per CTA, under a bound of `max_warps` per SM; ties go
// to 2, then 4, then 1.
inline int warps_per_cta_for_residency(size_t warp_bytes, size_t smem_sm, size_t reserved,
                                       int max_warps) {
  int best = 2, best_warps = -1;
  const int choices[3] = {2, 4, 1};
  for (int c = 0; c < 3; ++c) {
    const int rw = choices[c];
    int ctas = (int)(smem_sm / (rw * warp_bytes + reserved));
    if (ctas > max_warps / rw) ctas = max_warps / rw;
    if (ctas * rw > best_warps) {
      best_warps = ctas * rw;
      best = rw;
    }
  }
  return best;
}

}  // namespace lagp
