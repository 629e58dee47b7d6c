// Instantiations of the persistent batch kernel for block shapes of 512 threads (one translation
// unit per thread count, so that the shapes compile in parallel).
#include "block_dev.cuh"

namespace bp {

const void *batch_kernel_512_1() { return (const void *)k_batch<512, 1>; }
const void *batch_kernel_512_2() { return (const void *)k_batch<512, 2>; }

}  // namespace bp
