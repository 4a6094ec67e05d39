// rf_launch.cpp -- host helpers shared by the launchers.
#include <stdint.h>

#include "rf_internal.h"

// Vector (128-bit) loads need every column read to start at the same 16-byte
// phase; the first `head` events before the first aligned one are read with
// scalar loads.
void rf_vec_plan(const RfProgram& P, const void* events, int64_t stride, int elem_bytes,
                 int* vec, int64_t* head) {
  const uintptr_t base = reinterpret_cast<uintptr_t>(events);
  uintptr_t ph0 = 0;
  bool same = true;
  for (int c = 0; c < P.n_cols; ++c) {
    uintptr_t a = base + (uintptr_t)((int64_t)P.col_obs[c] * stride * (int64_t)elem_bytes);
    uintptr_t ph = a & 15u;
    if (c == 0) ph0 = ph;
    else if (ph != ph0) same = false;
  }
  if (same && (ph0 % (uintptr_t)elem_bytes) == 0) {
    *vec = 1;
    *head = (int64_t)(((16u - ph0) & 15u) / (uintptr_t)elem_bytes);
  } else {
    *vec = 0;
    *head = 0;
  }
}
