/*
 * sped_probe.h -- measurement library of the benchmark (libsped_probe.so), not part of the
 * libsped C ABI and not on the solver path.
 *
 * sped_probe_gather replays the chain step's access stream without its arithmetic, to compare
 * the step with the rate at which the GPU serves the same random row gathers. X and Y: n x k
 * BF16 blocks with ld * 2 a multiple of 16 bytes and 16-byte aligned bases (the chain's
 * storage); Y receives, per row, the sum of the gathered 16-byte chunks (whole chunks are
 * written, row padding included). mode 0: the rows named by the CSR (col_idx read as the chain
 * step reads it); 1: as many rows per node, hashed uniformly from (entry index, seed), no index
 * stream; 2: as many consecutive rows r+1, r+2, ... (every warp request coalesced). Returns 0, or 1 (bad argument), 2 (k > 256),
 * 3 (launch error). Stream-ordered.
 */
#ifndef SPED_PROBE_H
#define SPED_PROBE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

int sped_probe_gather(int64_t n, const int32_t *d_row_ptr, const int32_t *d_col_idx, int k,
                      const void *d_X, int ldx, void *d_Y, int ldy, int mode, uint64_t seed,
                      void *stream);

#ifdef __cplusplus
}
#endif

#endif
