// Rasteriser instantiation for a per-pixel sorter of capacity K = 8.
#include "lr_raster.cuh"
LR_DEFINE_RASTER(8)
