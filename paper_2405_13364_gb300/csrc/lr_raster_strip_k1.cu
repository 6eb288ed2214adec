// Rasteriser instantiation with per-strip shared set-up for a per-pixel sorter of capacity K = 1.
#include "lr_raster_strip.cuh"
LR_DEFINE_RASTER_STRIP(1)
