// Serving loop: placeholder until the scheduler lands.
#include "fk_internal.h"

using namespace fk;
extern "C" {
int fk_serve_create(size_t, int, fk_server **) { return fail(FK_EUNSUPPORTED, "serving not built yet"); }
int fk_serve_add_table(fk_server *, fk_table *, int *) { return fail(FK_EUNSUPPORTED, "serving not built yet"); }
int fk_serve_submit(fk_server *, int, const void *, int, int, uint64_t *) { return fail(FK_EUNSUPPORTED, "serving not built yet"); }
int fk_serve_poll(fk_server *, uint64_t, void *, int *) { return fail(FK_EUNSUPPORTED, "serving not built yet"); }
int fk_serve_wait(fk_server *, uint64_t, void *, int) { return fail(FK_EUNSUPPORTED, "serving not built yet"); }
int fk_serve_stats(const fk_server *, uint64_t *, uint64_t *, uint64_t *, size_t *, int *) { return fail(FK_EUNSUPPORTED, "serving not built yet"); }
int fk_serve_destroy(fk_server *) { return FK_OK; }
}
