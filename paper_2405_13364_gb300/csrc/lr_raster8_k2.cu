// Rasteriser instantiation with 8x8-pixel blocks for a per-pixel sorter of capacity K = 2.
#include "lr_raster8.cuh"
LR_DEFINE_RASTER8(2)
