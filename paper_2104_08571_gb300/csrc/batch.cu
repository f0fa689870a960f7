// Batched and served execution (filled in by the batch runtime).
#include "runtime.h"

void batch_runtime_destroy(ripple_ctx) {}
