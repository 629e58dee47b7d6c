// Instantiations of the persistent batch kernel for block shapes of 256 threads (one translation
// unit per thread count, so that the shapes compile in parallel).
#include "block_dev.cuh"

namespace bp {

const void *batch_kernel_256_1() { return (const void *)k_batch<256, 1>; }
const void *batch_kernel_256_2() { return (const void *)k_batch<256, 2>; }
const void *batch_kernel_256_4() { return (const void *)k_batch<256, 4>; }

}  // namespace bp
