// Pseudo-spectral (PSTD) field solver of a context (internal header).
#pragma once

#include <cstdint>

#include "mln.h"

struct mln_ctx;

namespace mln {

// Tables (twiddles, spectral multipliers) and work arrays of a periodic
// context with a power-of-two number of cells, in one device allocation.
mln_status pstd_init(mln_ctx *c);
void pstd_free(mln_ctx *c);
// n_steps steps from the context's buffer set 0, in place; src as for mln_step.
mln_status pstd_steps(mln_ctx *c, int64_t n_steps, const double *src);
// Kernel launches per time step (cell kernel + FFT passes).
int pstd_launches_per_step(int64_t n_cells, int64_t n_medium);

}  // namespace mln
