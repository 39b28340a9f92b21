/*
 * Seeded synthetic geometry for porous-media lattice Boltzmann workloads.
 *
 * This file holds no lattice Boltzmann arithmetic. It only decides which
 * lattice nodes are solid, so that the CUDA solver and the CPU oracle can be
 * fed the same inputs.
 *
 * Random numbers: splitmix64 (Steele, Lea and Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014), as its published definition
 * gives it. A double in [0,1) takes the top 53 bits of one output.
 *
 * Medium: overlapping solid spheres of one radius r, whose centres are
 * uniform real points in [0,nx)x[0,ny)x[0,nz). A node at integer
 * coordinates (x,y,z) is solid when its periodic minimum-image squared
 * distance to some centre is <= r^2. Spheres are added one at a time until
 * porosity (fluid nodes / all nodes) is <= the target; the sphere that
 * crosses the target is kept and the porosity reached is reported. This is
 * the paper's randomly placed overlapping spheres (Section 4.3), with the
 * stopping rule fixed here.
 *
 * Layout of every mask: uint8, index x + nx*(y + ny*z), 1 = solid.
 */
#include <stdint.h>
#include <stddef.h>
#include <math.h>

static uint64_t splitmix64_next(uint64_t* state)
{
    uint64_t z = (*state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static double uniform01(uint64_t* state)
{
    return (double)(splitmix64_next(state) >> 11) * (1.0 / 9007199254740992.0);
}

/* Smallest periodic image distance along one axis of length n. */
static double min_image(double d, int n)
{
    double h = 0.5 * (double)n;
    while (d > h) d -= (double)n;
    while (d < -h) d += (double)n;
    return d;
}

/*
 * Marks the nodes of one sphere solid. Returns how many nodes turned from
 * fluid to solid. The bounding box is scanned with wrapped indices, so a
 * sphere near a face continues on the opposite face. When the box is wider
 * than the domain on an axis, each node of that axis is visited once and the
 * minimum-image distance decides.
 */
static int64_t stamp_sphere(uint8_t* mask, int nx, int ny, int nz,
                            double cx, double cy, double cz, double r)
{
    int64_t added = 0;
    double r2 = r * r;
    int ext = (int)ceil(r) + 1;
    int x0 = (int)floor(cx) - ext, x1 = (int)floor(cx) + ext;
    int y0 = (int)floor(cy) - ext, y1 = (int)floor(cy) + ext;
    int z0 = (int)floor(cz) - ext, z1 = (int)floor(cz) + ext;
    if (x1 - x0 + 1 > nx) { x0 = 0; x1 = nx - 1; }
    if (y1 - y0 + 1 > ny) { y0 = 0; y1 = ny - 1; }
    if (z1 - z0 + 1 > nz) { z0 = 0; z1 = nz - 1; }
    for (int zz = z0; zz <= z1; ++zz) {
        int z = ((zz % nz) + nz) % nz;
        double dz = min_image((double)z - cz, nz);
        for (int yy = y0; yy <= y1; ++yy) {
            int y = ((yy % ny) + ny) % ny;
            double dy = min_image((double)y - cy, ny);
            double dyz = dy * dy + dz * dz;
            if (dyz > r2) continue;
            for (int xx = x0; xx <= x1; ++xx) {
                int x = ((xx % nx) + nx) % nx;
                double dx = min_image((double)x - cx, nx);
                if (dx * dx + dyz <= r2) {
                    size_t i = (size_t)x + (size_t)nx * ((size_t)y + (size_t)ny * (size_t)z);
                    if (!mask[i]) { mask[i] = 1; ++added; }
                }
            }
        }
    }
    return added;
}

/*
 * Fills mask (zeroed here first) with overlapping spheres until porosity
 * <= target_porosity or max_spheres spheres were placed.
 * out_info[0] = porosity reached, out_info[1] = spheres placed.
 * Returns 0, or -1 on bad arguments.
 */
int lbmin_sphere_pack(uint8_t* mask, int nx, int ny, int nz, double radius,
                      double target_porosity, uint64_t seed, int64_t max_spheres,
                      double* out_info)
{
    if (!mask || nx <= 0 || ny <= 0 || nz <= 0 || !(radius >= 0.0)) return -1;
    size_t n = (size_t)nx * (size_t)ny * (size_t)nz;
    for (size_t i = 0; i < n; ++i) mask[i] = 0;
    uint64_t state = seed;
    int64_t solid = 0, placed = 0;
    double phi = 1.0;
    while (phi > target_porosity && placed < max_spheres) {
        double cx = uniform01(&state) * (double)nx;
        double cy = uniform01(&state) * (double)ny;
        double cz = uniform01(&state) * (double)nz;
        solid += stamp_sphere(mask, nx, ny, nz, cx, cy, cz, radius);
        ++placed;
        phi = (double)((int64_t)n - solid) / (double)n;
    }
    if (out_info) { out_info[0] = phi; out_info[1] = (double)placed; }
    return 0;
}

/* Raw splitmix64 stream, for seeded initial fields in tests. */
void lbmin_splitmix64_fill(uint64_t seed, uint64_t* out, int64_t count)
{
    uint64_t state = seed;
    for (int64_t i = 0; i < count; ++i) out[i] = splitmix64_next(&state);
}
