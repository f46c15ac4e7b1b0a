// Serving loop: placeholder until the request scheduler is in place.
#include "serve.h"

namespace gb {

void server_destroy(gf_handle_s* h) { (void)h; }

}  // namespace gb
