/*
 * synth.c -- seeded synthetic tomography slices for the MRF region-labelling
 * tests and benchmarks.
 *
 * This module generates INPUTS only: a phase map of random disks, a noisy FP64
 * intensity image drawn from it, and a jittered-grid Voronoi oversegmentation
 * (the region id of every pixel).  It holds none of the segmentation method's
 * arithmetic (no region means, no graph, no energies).  Both the CPU oracle and
 * the CUDA path consume exactly the arrays produced here.
 *
 * The paper evaluates on two stacks that are not available here (a synthetic
 * porous-media benchmark corrupted with noise, and a beamline experiment;
 * Section 4.1.1); these slices stand in for them: two- or three-phase images
 * of overlapping disks plus additive Gaussian noise, oversegmented into
 * compact convex superpixels, which is the kind of input Section 3.1 describes
 * (an irregular partition into non-overlapping regions).
 *
 * Random numbers: SplitMix64 (Steele, Lea, Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014), uniform doubles from the top
 * 53 bits, normals by the Box-Muller transform.  Each part of a slice (disks,
 * Voronoi seeds, pitch, noise) draws from its own stream derived from the slice
 * seed, so the parts are independent of one another's draw counts.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int64_t height, width;
    int32_t n_phases;      /* 2 or 3 */
    int32_t pad0;
    double phase_mu[3];    /* intensity of each phase */
    double noise_sigma;    /* additive Gaussian noise std */
    double r_min, r_max;   /* disk radius range, U[r_min, r_max] */
    double area_frac;      /* 2 phases: total covered fraction; 3 phases: new
                              coverage of each disk family */
    double pitch_min, pitch_max; /* Voronoi grid pitch, U[min, max] (equal => fixed) */
    double jitter;         /* seed jitter, U[-jitter, jitter] on each axis */
    uint64_t seed;
} synth_cfg;

typedef struct { uint64_t s; } sm64;

static uint64_t sm64_next(sm64* g) {
    uint64_t z = (g->s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
/* uniform in [0, 1) */
static double sm64_unif(sm64* g) { return (double)(sm64_next(g) >> 11) * 0x1.0p-53; }

static sm64 stream_for(uint64_t seed, uint64_t part) {
    sm64 g;
    g.s = seed * 0xD1B54A32D192ED03ull + part * 0x8CB92BA72F3D8DD7ull + 0x632BE59BD9B4E019ull;
    (void)sm64_next(&g);
    return g;
}

/* Paint disks of value `phase` into `truth` until the number of pixels newly
 * set to `phase` reaches `target`.  Returns the number of disks drawn. */
static int64_t paint_family(uint8_t* truth, int64_t H, int64_t W, sm64* g, double rmin,
                            double rmax, uint8_t phase, int64_t target) {
    int64_t covered = 0, ndisk = 0;
    while (covered < target) {
        double cx = sm64_unif(g) * (double)W;
        double cy = sm64_unif(g) * (double)H;
        double r = rmin + (rmax - rmin) * sm64_unif(g);
        int64_t r0 = (int64_t)floor(cy - r), r1 = (int64_t)ceil(cy + r);
        int64_t c0 = (int64_t)floor(cx - r), c1 = (int64_t)ceil(cx + r);
        if (r0 < 0) r0 = 0;
        if (c0 < 0) c0 = 0;
        if (r1 > H - 1) r1 = H - 1;
        if (c1 > W - 1) c1 = W - 1;
        for (int64_t rr = r0; rr <= r1; ++rr) {
            double dy = (double)rr + 0.5 - cy;
            for (int64_t cc = c0; cc <= c1; ++cc) {
                double dx = (double)cc + 0.5 - cx;
                if (dx * dx + dy * dy <= r * r) {
                    uint8_t* t = &truth[rr * W + cc];
                    if (*t != phase) {
                        *t = phase;
                        ++covered;
                    }
                }
            }
        }
        ++ndisk;
        if (ndisk > 100000000) break; /* unreachable for sane configs */
    }
    return ndisk;
}

/*
 * Generate one slice.  image: f64[H*W], region_ids: i32[H*W] (raw Voronoi seed
 * index; cells that receive no pixel leave gaps in the id range), truth:
 * u8[H*W] phase map.  Returns the Voronoi pitch used (>0) or a negative value
 * on bad arguments.
 */
double synth_slice(const synth_cfg* cfg, double* image, int32_t* region_ids, uint8_t* truth) {
    const int64_t H = cfg->height, W = cfg->width;
    if (H <= 0 || W <= 0 || cfg->n_phases < 2 || cfg->n_phases > 3) return -1.0;
    const int64_t N = H * W;
    memset(truth, 0, (size_t)N);

    /* phase map */
    sm64 gd = stream_for(cfg->seed, 1);
    if (cfg->n_phases == 2) {
        paint_family(truth, H, W, &gd, cfg->r_min, cfg->r_max, 1,
                     (int64_t)ceil(cfg->area_frac * (double)N));
    } else {
        paint_family(truth, H, W, &gd, cfg->r_min, cfg->r_max, 1,
                     (int64_t)ceil(cfg->area_frac * (double)N));
        paint_family(truth, H, W, &gd, cfg->r_min, cfg->r_max, 2,
                     (int64_t)ceil(cfg->area_frac * (double)N));
    }

    /* Voronoi seeds on a jittered grid */
    sm64 gp = stream_for(cfg->seed, 2);
    double p = cfg->pitch_min;
    if (cfg->pitch_max > cfg->pitch_min) p = cfg->pitch_min + (cfg->pitch_max - cfg->pitch_min) * sm64_unif(&gp);
    const double J = cfg->jitter;
    const int64_t nx = (int64_t)ceil((double)W / p), ny = (int64_t)ceil((double)H / p);
    if (nx * ny > 2147483647ll) return -2.0;
    double* sx = (double*)malloc(sizeof(double) * (size_t)(nx * ny));
    double* sy = (double*)malloc(sizeof(double) * (size_t)(nx * ny));
    if (!sx || !sy) { free(sx); free(sy); return -3.0; }
    sm64 gs = stream_for(cfg->seed, 3);
    for (int64_t j = 0; j < ny; ++j)
        for (int64_t i = 0; i < nx; ++i) {
            double jx = (2.0 * sm64_unif(&gs) - 1.0) * J;
            double jy = (2.0 * sm64_unif(&gs) - 1.0) * J;
            sx[j * nx + i] = ((double)i + 0.5) * p + jx;
            sy[j * nx + i] = ((double)j + 0.5) * p + jy;
        }

    /* nearest seed per pixel centre; ties go to the lower seed index.  Rings of
     * grid cells are searched outward until no unsearched cell can hold a seed
     * at least as close as the best one found: a seed of a cell R rings away is
     * at least (R - 1/2) p - J from any pixel of the centre cell. */
    for (int64_t r = 0; r < H; ++r) {
        const double py = (double)r + 0.5;
        int64_t j0 = (int64_t)floor(py / p);
        if (j0 >= ny) j0 = ny - 1;
        for (int64_t c = 0; c < W; ++c) {
            const double px = (double)c + 0.5;
            int64_t i0 = (int64_t)floor(px / p);
            if (i0 >= nx) i0 = nx - 1;
            double best = INFINITY;
            int64_t bidx = -1;
            for (int64_t R = 0;; ++R) {
                double lb = ((double)R - 0.5) * p - J;
                if (R > 0 && lb > 0.0 && best < lb * lb) break;
                if (R > 0 && i0 - R < 0 && j0 - R < 0 && i0 + R >= nx && j0 + R >= ny) break;
                for (int64_t dj = -R; dj <= R; ++dj) {
                    int64_t j = j0 + dj;
                    if (j < 0 || j >= ny) continue;
                    for (int64_t di = -R; di <= R; ++di) {
                        if (dj != -R && dj != R && di != -R && di != R) continue; /* ring only */
                        int64_t i = i0 + di;
                        if (i < 0 || i >= nx) continue;
                        int64_t s = j * nx + i;
                        double ddx = px - sx[s], ddy = py - sy[s];
                        double d2 = ddx * ddx + ddy * ddy;
                        if (d2 < best || (d2 == best && s < bidx)) {
                            best = d2;
                            bidx = s;
                        }
                    }
                }
            }
            region_ids[r * W + c] = (int32_t)bidx;
        }
    }
    free(sx);
    free(sy);

    /* intensities: phase mean plus Gaussian noise (Box-Muller pairs, row-major) */
    sm64 gn = stream_for(cfg->seed, 4);
    const double two_pi = 6.283185307179586476925286766559;
    for (int64_t k = 0; k < N; k += 2) {
        double u1 = 1.0 - sm64_unif(&gn); /* (0, 1] */
        double u2 = sm64_unif(&gn);
        double rad = sqrt(-2.0 * log(u1));
        double z0 = rad * cos(two_pi * u2), z1 = rad * sin(two_pi * u2);
        image[k] = cfg->phase_mu[truth[k]] + cfg->noise_sigma * z0;
        if (k + 1 < N) image[k + 1] = cfg->phase_mu[truth[k + 1]] + cfg->noise_sigma * z1;
    }
    return p;
}
