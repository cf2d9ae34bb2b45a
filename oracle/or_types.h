/* Shared types of the FP64 oracle's C sources (test infrastructure only). */
#ifndef OR_TYPES_H
#define OR_TYPES_H

typedef struct {
    int kind, nx, ny, nz;
    double dx, dy, dz, cx, cy, cz, sid, sdd;
    int n_views, views_per_rotation;
    double start_angle, feed, z_start;
    int n_rows;
    double row_pitch;
    int n_channels;
    double channel_pitch, channel_offset, row_offset;
} or_geometry;

typedef struct {
    int n_e;
    const double *I0;     /* [2][n_e] */
    const double *mu;     /* [2][n_e] */
    const double *bowtie; /* [n_channels] or NULL (== 1) */
} or_model;

typedef struct {
    long idx;  /* voxel index iz*ny*nx + iy*nx + ix */
    double w;  /* h(x, y) in mm */
} or_tap;

int or_ray_taps(const or_geometry *g, long v, int r, int k, or_tap *T);
int or_max_taps(const or_geometry *g);
void or_forward(const or_geometry *g, const double *c, double *l, int v0, int v1);

#endif
