// lr_serve.h -- internal link between the context (lr_api.cu) and the serving loop
// (lr_serve.cu).
#pragma once

#include "lr.h"

struct lr_server;

// the context's server pointer (nullptr when no server runs)
lr_server** lr_internal_server_slot(lr_ctx* ctx);
// the configuration the context was created with (defaults filled in)
const lr_config* lr_internal_config(const lr_ctx* ctx);
// the context's light (unit direction toward the light, ambient) for lit views
const float* lr_internal_light(const lr_ctx* ctx);
// argument checks of one view, as lr_render_batch applies them (no GPU work)
lr_status lr_internal_check_view(lr_ctx* ctx, const lr_view* view);
// programmatic dependent launch for the context's next renders: -1 as its flags say, 0 off,
// 1 on (the server turns it on for a batch that runs alone on the GPU)
void lr_internal_set_pdl(lr_ctx* ctx, int pdl);
