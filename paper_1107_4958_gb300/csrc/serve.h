// Serving loop (serve.cpp): continuous batching of filter requests.
#pragma once

#include "internal.h"

namespace gb {

void server_destroy(gf_handle_s* h);

}  // namespace gb
