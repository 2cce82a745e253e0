// Launch helpers of the tile operator kernel (tpt_tile.cuh): tile size,
// CTA size and grid, shared by the FP32, BF16-storage and FP64 translation
// units.
#pragma once

#include <algorithm>

#include "internal.h"
#include "tpt_tile.cuh"

namespace hdg {

#define TILE_N_SWITCH(n, CALL)                                                  \
  switch (n) {                                                                  \
    case 2: return CALL(2); case 3: return CALL(3); case 4: return CALL(4);     \
    case 5: return CALL(5); case 6: return CALL(6); case 7: return CALL(7);     \
    case 8: return CALL(8); case 9: return CALL(9); case 10: return CALL(10);   \
    case 11: return CALL(11); case 12: return CALL(12); case 13: return CALL(13); \
    case 14: return CALL(14); case 15: return CALL(15); case 16: return CALL(16); \
    case 17: return CALL(17);                                                   \
    default: break;                                                             \
  }

template <typename T, int N>
size_t tile_smem_bytes(int E) {
  return sizeof(T) * (size_t)E * tile_smem_per_elem<T, N>();
}

// resident CTAs per SM of tpt_tile_kernel<T, ST, N, DZM> with `rounds`
// elements per thread (tiles of G x rounds elements; 0 if it cannot run)
template <typename T, typename ST, int N, int DZM, int CGM>
int tile_occupancy(int rounds) {
  static int cached[8] = {0};
  const int G = tile_groups(N);
  if (rounds < 1 || rounds > tile_rounds<T, CGM>() || G * rounds > kTileMaxE) return 0;
  if (cached[rounds] != 0) return std::max(cached[rounds], 0);
  const size_t smem = tile_smem_bytes<T, N>(G * rounds);
  int nb = 0;
  if (smem > 227 * 1024 ||
      cudaFuncSetAttribute(tpt_tile_kernel<T, ST, N, DZM, CGM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)std::max(smem, kSmemOptIn)) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, tpt_tile_kernel<T, ST, N, DZM, CGM>, tile_cta_threads(N), smem) !=
          cudaSuccess) {
    cudaGetLastError();
    nb = 0;
  }
  cached[rounds] = nb > 0 ? nb : -1;
  return nb;
}

// Rounds for nelem elements and nrhs right-hand sides on `sms` SMs: the one
// that minimises the elements one thread processes in sequence (tiles per
// resident CTA, rounded up, times the rounds plus a per-tile overhead of
// half an element's worth), the larger on ties.
template <typename T, typename ST, int N, int DZM, int CGM>
int tile_pick(long long nelem, int nrhs, int sms) {
  const int G = tile_groups(N);
  int best = 1;
  double best_cost = -1.0;
  for (int r = 1; r <= tile_rounds<T, CGM>(); ++r) {
    const int occ = tile_occupancy<T, ST, N, DZM, CGM>(r);
    if (occ < 1) continue;
    const long long E = (long long)G * r;
    const long long tiles = (nelem + E - 1) / E * nrhs;
    const long long resident = (long long)sms * occ;
    const double cost = (double)((tiles + resident - 1) / resident) * (r + 0.5);
    if (best_cost < 0.0 || cost <= best_cost) {
      best_cost = cost;
      best = r;
    }
  }
  return best;
}

// Launch over all elements of nrhs right-hand sides.  `E` > 0 asks for tiles
// of about E elements (rounded to a multiple of G; reduced to what fits),
// else tile_pick.  Sets a.seg = E and a.ppb = G.  The grid is one resident
// wave (at most) of CTAs per right-hand side row, each looping over tiles.
template <typename T, typename ST, int N, int DZM, int CGM>
cudaError_t tile_launch(TptArgs<T, ST> a, int nrhs, int sms, int E, cudaStream_t s) {
  const long long nelem = (long long)a.mesh.ne[0] * a.mesh.ne[1] * a.mesh.ne[2];
  if (nelem <= 0) return cudaSuccess;
  const int G = tile_groups(N);
  int rounds = E > 0 ? std::max(1, (E + G - 1) / G) : tile_pick<T, ST, N, DZM, CGM>(nelem, nrhs, sms);
  rounds = std::min(rounds, tile_rounds<T, CGM>());
  while (rounds > 1 && tile_occupancy<T, ST, N, DZM, CGM>(rounds) < 1) --rounds;
  const int occ = tile_occupancy<T, ST, N, DZM, CGM>(rounds);
  if (occ < 1) return cudaErrorInvalidConfiguration;
  a.seg = G * rounds;
  a.ppb = G;
  const long long tiles = (nelem + a.seg - 1) / a.seg;
  const long long resident = (long long)sms * occ;
  const long long per_rhs = std::max(1LL, resident / std::max(nrhs, 1));
  const unsigned gx = (unsigned)std::min(tiles, per_rhs);
  const size_t smem = tile_smem_bytes<T, N>(a.seg);
  const dim3 grid(gx, (unsigned)nrhs), block((unsigned)tile_cta_threads(N));
  if (CGM == 2 || a.pdl) {
    // the persistent kernel needs every CTA resident (cooperative launch: the
    // launch fails rather than runs if the grid cannot be co-resident)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    if (CGM == 2) {
      attr[0].id = cudaLaunchAttributeCooperative;
      attr[0].val.cooperative = 1;
    } else {
      attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
      attr[0].val.programmaticStreamSerializationAllowed = 1;
    }
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, tpt_tile_kernel<T, ST, N, DZM, CGM>, a);
  }
  tpt_tile_kernel<T, ST, N, DZM, CGM><<<grid, block, smem, s>>>(a);
  return cudaGetLastError();
}

// D_Z^-1 source of the tile kernel: no table -> computed in the kernel;
// one element class -> the table row in registers; else the element's table.
// a.cg selects the fused CG step (FP32 and FP64 storage only).
template <typename T, typename ST, int N, int CGM>
cudaError_t tile_dispatch_dz_cg(const TptArgs<T, ST>& a, int nrhs, int sms, int E, cudaStream_t s) {
  if (a.dinv == nullptr) {
    // FP64 always reads a table (a division costs more FP64-pipe time than the load)
    if constexpr (sizeof(T) == 8) return cudaErrorInvalidValue;
    else return tile_launch<T, ST, N, 1, CGM>(a, nrhs, sms, E, s);
  }
  if (a.mesh.uniform) return tile_launch<T, ST, N, 0, CGM>(a, nrhs, sms, E, s);
  return tile_launch<T, ST, N, 2, CGM>(a, nrhs, sms, E, s);
}

template <typename T, typename ST, int N>
cudaError_t tile_dispatch_dz(const TptArgs<T, ST>& a, int nrhs, int sms, int E, cudaStream_t s) {
  if constexpr (std::is_same<T, ST>::value) {
    if (a.cg == 1) return tile_dispatch_dz_cg<T, ST, N, 1>(a, nrhs, sms, E, s);
    if (a.cg == 2) return tile_dispatch_dz_cg<T, ST, N, 2>(a, nrhs, sms, E, s);
  }
  if (a.cg) return cudaErrorInvalidValue;
  return tile_dispatch_dz_cg<T, ST, N, 0>(a, nrhs, sms, E, s);
}

}  // namespace hdg
