// Half-storage instances of the persistent batch iteration (see
// batch_persist.cu).
#include "batch_persist.cuh"

namespace lfsr {

using PersistKernel = void (*)(const Geom, const Geom, const Geom, const PersistArgs*,
                               unsigned long long*);

PersistKernel persist_kernel_f16(int WR, int PR, int Z0, int K0, int Z1, int K1) {
#define LFSR_PERSIST_PICK_H(wr, pr, z0, k0, z1, k1)                          \
  if (WR == wr && PR == pr && Z0 == z0 && K0 == k0 && Z1 == z1 && K1 == k1) \
    return k_batch_iter<__half, wr, pr, z0, k0, z1, k1>;
  LFSR_PERSIST_PICK_H(2, 1, 2, 5, 0, 0)
  LFSR_PERSIST_PICK_H(3, 1, 2, 7, 0, 0)
  LFSR_PERSIST_PICK_H(3, 1, 3, 9, 0, 0)
  LFSR_PERSIST_PICK_H(3, 1, 2, 7, 3, 9)
#undef LFSR_PERSIST_PICK_H
  return nullptr;
}

}  // namespace lfsr
