// br_h1.cu -- blind-rotation kernel shapes with H = 1 (2H warps per gate); gadget length L = 3 and 2.
#include "br_kernel.cuh"

namespace arx {

cudaError_t launch_br_h1(const BrArgs &args, int GT, int L, int grid, cudaStream_t st) {
  if (L == 2) {
    switch (GT) {
      case 1: return br::launch_shape<1, 1, 2>(args, grid, st);
      case 2: return br::launch_shape<1, 2, 2>(args, grid, st);
      case 4: return br::launch_shape<1, 4, 2>(args, grid, st);
      case 6: return br::launch_shape<1, 6, 2>(args, grid, st);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (GT) {
    case 1: return br::launch_shape<1, 1, 3>(args, grid, st);
    case 2: return br::launch_shape<1, 2, 3>(args, grid, st);
    case 4: return br::launch_shape<1, 4, 3>(args, grid, st);
    case 6: return br::launch_shape<1, 6, 3>(args, grid, st);
    default: return cudaErrorInvalidValue;
  }
}

size_t br_smem_h1(int GT, int L) {
  if (L == 2) {
    switch (GT) {
      case 1: return br::br_smem_bytes<1, 1, 2>();
      case 2: return br::br_smem_bytes<1, 2, 2>();
      case 4: return br::br_smem_bytes<1, 4, 2>();
      case 6: return br::br_smem_bytes<1, 6, 2>();
      default: return 0;
    }
  }
  switch (GT) {
    case 1: return br::br_smem_bytes<1, 1>();
    case 2: return br::br_smem_bytes<1, 2>();
    case 4: return br::br_smem_bytes<1, 4>();
    case 6: return br::br_smem_bytes<1, 6>();
    default: return 0;
  }
}

int br_occupancy_h1(int GT, int L) {
  if (L == 2) {
    switch (GT) {
      case 1: return br::occupancy_shape<1, 1, 2>();
      case 2: return br::occupancy_shape<1, 2, 2>();
      case 4: return br::occupancy_shape<1, 4, 2>();
      case 6: return br::occupancy_shape<1, 6, 2>();
      default: return 0;
    }
  }
  switch (GT) {
    case 1: return br::occupancy_shape<1, 1, 3>();
    case 2: return br::occupancy_shape<1, 2, 3>();
    case 4: return br::occupancy_shape<1, 4, 3>();
    case 6: return br::occupancy_shape<1, 6, 3>();
    default: return 0;
  }
}

}  // namespace arx
