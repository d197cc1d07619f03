/* The C ABI used from plain C99 (no C++, no Python): both headers compile
 * with warnings as errors, and the host-side calls that need no GPU behave
 * as include/fdtd.h states.  Built and run by tests/test_c_abi.py. */
#include <stdio.h>
#include <string.h>

#include "fdtd.h"
#include "fdtd_mlp.h"

#define CHECK(x)                                               \
    do {                                                       \
        if (!(x)) {                                            \
            printf("FAIL line %d: %s\n", __LINE__, #x);        \
            return 1;                                          \
        }                                                      \
    } while (0)

enum { NX = 16, NY = 14, NZ = 12 };

int main(void)
{
    static uint8_t cm[NX * NY * NZ];
    fdtd_material mats[2] = {{1.0, 0.0, 1.0}, {10.0, 0.01, 1.0}};
    fdtd_cpml cp = {3, 3.0, 1.0, 0.0, 1.0, 0.0};
    fdtd_grid *g = NULL;
    int id = -1, ns = 0, nn = 0, q;
    double lim = 0.0;
    size_t bytes = 0, bytes_cpml = 0;

    CHECK(fdtd_create_grid(NX, NY, NZ, 0.1, 1.5, NULL, NULL, &g) == FDTD_ECOURANT && g == NULL);
    CHECK(fdtd_create_grid(1, NY, NZ, 0.1, 0.9, NULL, NULL, &g) == FDTD_EINVAL && g == NULL);
    CHECK(fdtd_create_grid(NX, NY, NZ, 0.1, 0.9, NULL, NULL, &g) == FDTD_OK && g != NULL);
    for (q = 0; q < NX * NY * NZ / 2; ++q) cm[q] = 1;          /* lower half (k < NZ/2): soil */
    CHECK(fdtd_set_materials(g, cm, mats, 2) == FDTD_OK);
    CHECK(fdtd_add_wire(g, 5, 6, 2, 5, 6, 8, 0.004, &id) == FDTD_OK && id == 0);
    CHECK(fdtd_add_wire(g, 5, 6, 2, 5, 7, 8, 0.004, NULL) == FDTD_EINVAL);   /* not along one axis */
    CHECK(strlen(fdtd_last_error(g)) > 0);
    CHECK(fdtd_add_oblique_wire(g, 5.0, 6.0, 8.0, 11.3, 9.2, 10.1, 0.002, &id) == FDTD_OK && id == 0);
    CHECK(fdtd_wire_counts(g, &ns, &nn) == FDTD_OK && ns == 7 && nn == ns + 1);
    CHECK(fdtd_wire_courant_limit(g, &lim) == FDTD_OK && lim > 0.5 && lim <= 1.0);
    CHECK(fdtd_add_probe(g, FDTD_PROBE_V, 5, 6, 1, 2, 1, &id) == FDTD_OK && id == 0);
    CHECK(fdtd_add_probe(g, 9, 5, 6, 1, 2, 1, NULL) == FDTD_EINVAL);
    CHECK(fdtd_arena_bytes(g, 100, &bytes) == FDTD_OK && bytes >= (size_t)6 * NX * NY * NZ * 4);
    fdtd_destroy(g);

    g = NULL;
    CHECK(fdtd_create_grid(NX, NY, NZ, 0.1, 0.9, &cp, NULL, &g) == FDTD_OK);
    CHECK(fdtd_arena_bytes(g, 100, &bytes_cpml) == FDTD_OK && bytes_cpml > bytes);
    fdtd_destroy(g);
    fdtd_destroy(NULL);
    printf("ok %d %d %.4f %lu %lu\n", ns, nn, lim, (unsigned long)bytes, (unsigned long)bytes_cpml);
    return 0;
}
