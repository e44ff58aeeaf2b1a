// Phase-B training kernels for S = 3 live-range warps, extended instantiations.
#define APSM_CHUNK_S 3
#define APSM_CHUNK_EXT 1
#include "train_chunk_inst.cuh"
