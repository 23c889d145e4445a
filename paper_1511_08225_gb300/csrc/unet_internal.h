// unet_internal.h -- what the 2D path uses of the U-Net beyond its C ABI: the
// forward pass on a caller's stream and the network's grid.
#pragma once

#include <cuda_runtime.h>

#include "slpic_unet.h"

// slpic_unet_forward on `stream` (the handle's own stream is left alone).
int slpic_unet_forward_on(slpic_unet_t *h, int nb, const float *x, float *y, cudaStream_t stream);
// Grid and batch capacity of the network.
void slpic_unet_shape(const slpic_unet_t *h, int *height, int *width, int *max_batch);
