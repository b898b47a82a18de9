/*
 * G-VOM per-scan voxel map update -- CPU ORACLE (test infrastructure only).
 *
 * This file is the plain, slow, single-threaded FP64 statement of what the
 * map update computes. It exists so that tests, the smoke check and the CPU
 * baseline leg of the benchmark can check the CUDA library against it. The
 * product path never links, loads or calls it, and it shares no code,
 * header, table or helper with the CUDA library.
 *
 * Every function follows the paper (G-VOM, Overbye & Saripalli, arXiv
 * 2109.13176) section it cites; where the paper is silent the reading used is
 * stated next to the code. Build with -ffp-contract=off: every FP64 operation
 * below is one IEEE round-to-nearest operation, in the order written, and
 * fma() is the correctly rounded fused multiply-add of C99.
 *
 * State layout (logical, window-relative, un-rotated):
 *   cell (ix, iy, iz), 0 <= ix < nx ..., linear index ((ix*ny)+iy)*nz+iz
 *   hits[V] u32, passes[V] u32, minz[V] f32 (+inf where empty)
 *   origin[3] int64 = world voxel index of window cell (0,0,0)
 * 2D outputs: [ix*ny + iy].
 *
 * Parity status of each function is listed at its definition.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int32_t nx, ny, nz;
    double res;          /* voxel edge, metres */
    double max_range;    /* rays longer than this are dropped, metres */
    float obs_min_h;     /* obstacle band above ground, metres */
    float obs_max_h;
    uint32_t hard_num;   /* hard iff density >= hard_num / hard_den */
    uint32_t hard_den;
    int32_t slope_n;     /* odd window edge N of the N x N plane fit */
    int32_t slope_min_px;/* defined pixels needed for a fit */
    int32_t neg_max_px;  /* cone search radius, pixels */
    float neg_thresh;    /* negative obstacle threshold on Delta H, metres */
} or_params;

typedef struct {
    int64_t points_in;      /* points offered */
    int64_t rays_valid;     /* points kept by the filter and quantiser */
    int64_t hits_in_window; /* valid points whose endpoint cell is in the window */
    int64_t pass_visits;    /* pass-count increments made */
} or_stats;

/* Quantised coordinates must stay below this magnitude (1/256-voxel units),
 * so that every product in the traversal fits in 64 bits. A ray whose sensor
 * or endpoint is further than 2^22 voxels from the window origin is dropped
 * (reading: the paper's maps are a few hundred voxels wide). */
#define OR_QLIM (1LL << 30)

static int64_t floor_div(int64_t a, int64_t b) /* b > 0 */
{
    int64_t q = a / b;
    if ((a % b) != 0 && a < 0) q -= 1;
    return q;
}

static int64_t lin(const or_params* p, int64_t ix, int64_t iy, int64_t iz)
{
    return (ix * p->ny + iy) * p->nz + iz;
}

static int in_window(const or_params* p, const int64_t c[3])
{
    return c[0] >= 0 && c[0] < p->nx && c[1] >= 0 && c[1] < p->ny && c[2] >= 0 && c[2] < p->nz;
}

/* Map origin for a vehicle position (Sec. III-A: the origin is an integer
 * multiple of the resolution; Sec. III-D: the combined map takes the newest
 * map's location). Reading: the window is centred on the vehicle voxel,
 * O = floor(vehicle / res) - (nx/2, ny/2, nz/2). Pinned by tests (exact
 * values for chosen positions). */
void or_origin_for_pose(const or_params* p, const double vehicle[3], int64_t out[3])
{
    const double inv_res = 1.0 / p->res;
    const int32_t half[3] = {p->nx / 2, p->ny / 2, p->nz / 2};
    for (int a = 0; a < 3; ++a)
        out[a] = (int64_t)floor(vehicle[a] * inv_res) - half[a];
}

/* Clear a map to the empty state: no hits, no passes, min height +inf. */
void or_clear(const or_params* p, uint32_t* hits, uint32_t* passes, float* minz)
{
    const int64_t V = (int64_t)p->nx * p->ny * p->nz;
    for (int64_t i = 0; i < V; ++i) {
        hits[i] = 0;
        passes[i] = 0;
        minz[i] = INFINITY;
    }
}

/* Window shift (Sec. III-A origin, Sec. III-D combination by index offset).
 * The map moves from origin old_o to new_o; a cell keeps its metrics when
 * its world voxel lies in both windows, cells entering the window start
 * empty, cells leaving are dropped. Pinned by tests: shift by zero is the
 * identity, shift(a) then shift(b) equals shift(a+b) on cells that stayed,
 * and a shift by the full window clears everything. */
void or_shift(const or_params* p, const int64_t old_o[3], const int64_t new_o[3],
              uint32_t* hits, uint32_t* passes, float* minz)
{
    const int64_t V = (int64_t)p->nx * p->ny * p->nz;
    uint32_t* h2 = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)V);
    uint32_t* p2 = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)V);
    float* m2 = (float*)malloc(sizeof(float) * (size_t)V);
    for (int64_t ix = 0; ix < p->nx; ++ix)
        for (int64_t iy = 0; iy < p->ny; ++iy)
            for (int64_t iz = 0; iz < p->nz; ++iz) {
                const int64_t dst = lin(p, ix, iy, iz);
                /* the same world voxel, in the old window's coordinates */
                int64_t j[3] = {new_o[0] + ix - old_o[0], new_o[1] + iy - old_o[1],
                                new_o[2] + iz - old_o[2]};
                if (in_window(p, j)) {
                    const int64_t src = lin(p, j[0], j[1], j[2]);
                    h2[dst] = hits[src];
                    p2[dst] = passes[src];
                    m2[dst] = minz[src];
                } else {
                    h2[dst] = 0;
                    p2[dst] = 0;
                    m2[dst] = INFINITY;
                }
            }
    memcpy(hits, h2, sizeof(uint32_t) * (size_t)V);
    memcpy(passes, p2, sizeof(uint32_t) * (size_t)V);
    memcpy(minz, m2, sizeof(float) * (size_t)V);
    free(h2);
    free(p2);
    free(m2);
}

/* ---------------------------------------------------------------------- */
/* Ray traversal (Sec. III-A: a voxel counts the rays that cross it;
 * Sec. III-C: every lidar ray is traced).
 *
 * Endpoints are integers in 1/256-voxel units relative to the window origin.
 * The segment P(t) = A + t (B - A), t in [0, 1], meets cell c iff for some t
 * every axis satisfies 256 c_i <= P_i(t) < 256 (c_i + 1) (half-open cells).
 * Written out as events: along an axis moving up, P_i reaches the boundary
 * 256 k at t = (256 k - A_i) / d_i and the new cell k holds from that t on;
 * along an axis moving down, P_i reaches 256 k at t = (A_i - 256 k) / |d_i|,
 * the old cell k still holds at that t and cell k - 1 holds just after it.
 * So at one t the upward crossings apply at t and the downward ones just
 * after it: the walk emits the cell after all upward crossings sharing t,
 * then the cell after all downward crossings sharing t.
 * Pinned by tests against a brute-force exact-rational test of every cell of
 * small grids. */

typedef struct {
    int64_t num, den; /* t = num / den, den > 0 */
    int axis;
    int dir;          /* +1 up, -1 down */
} or_event;

static int event_cmp(const void* pa, const void* pb)
{
    const or_event* a = (const or_event*)pa;
    const or_event* b = (const or_event*)pb;
    /* compare a.num/a.den with b.num/b.den exactly; |num|,|den| < 2^31 */
    const int64_t l = a->num * b->den, r = b->num * a->den;
    if (l != r) return l < r ? -1 : 1;
    if (a->dir != b->dir) return a->dir > b->dir ? -1 : 1; /* upward first */
    return a->axis - b->axis;
}

typedef void (*or_visit_fn)(void* ctx, const int64_t cell[3]);

/* Visit every cell of the traversal set, in order along the ray, start cell
 * first and endpoint cell last. */
static void or_traverse(const int64_t A[3], const int64_t B[3], or_visit_fn visit, void* ctx)
{
    int64_t c[3], ce[3];
    int64_t n_ev = 0;
    for (int a = 0; a < 3; ++a) {
        c[a] = floor_div(A[a], 256);
        ce[a] = floor_div(B[a], 256);
        n_ev += llabs(ce[a] - c[a]);
    }
    or_event* ev = (or_event*)malloc(sizeof(or_event) * (size_t)(n_ev > 0 ? n_ev : 1));
    int64_t m = 0;
    for (int a = 0; a < 3; ++a) {
        const int64_t d = B[a] - A[a];
        if (d > 0) {
            for (int64_t k = c[a] + 1; k <= ce[a]; ++k) {
                ev[m].num = 256 * k - A[a];
                ev[m].den = d;
                ev[m].axis = a;
                ev[m].dir = +1;
                ++m;
            }
        } else if (d < 0) {
            for (int64_t k = c[a]; k >= ce[a] + 1; --k) {
                ev[m].num = A[a] - 256 * k;
                ev[m].den = -d;
                ev[m].axis = a;
                ev[m].dir = -1;
                ++m;
            }
        }
    }
    qsort(ev, (size_t)m, sizeof(or_event), event_cmp);

    visit(ctx, c);
    int64_t i = 0;
    while (i < m) {
        /* the group of events sharing this t */
        int64_t j = i;
        while (j < m && ev[j].num * ev[i].den == ev[i].num * ev[j].den) ++j;
        int any_up = 0, any_down = 0;
        for (int64_t k = i; k < j; ++k)
            if (ev[k].dir > 0) { c[ev[k].axis] += 1; any_up = 1; }
        if (any_up) visit(ctx, c);
        for (int64_t k = i; k < j; ++k)
            if (ev[k].dir < 0) { c[ev[k].axis] -= 1; any_down = 1; }
        if (any_down) visit(ctx, c);
        i = j;
    }
    free(ev);
}

/* Collects the traversal in an array (used by the traversal pin tests). */
typedef struct {
    int64_t* out;
    int64_t cap, n;
} or_collect;

static void collect_visit(void* vctx, const int64_t cell[3])
{
    or_collect* ctx = (or_collect*)vctx;
    if (ctx->n < ctx->cap) {
        ctx->out[3 * ctx->n + 0] = cell[0];
        ctx->out[3 * ctx->n + 1] = cell[1];
        ctx->out[3 * ctx->n + 2] = cell[2];
    }
    ctx->n += 1;
}

/* Traversal of one segment, cells written to out[3*k..3*k+2]; returns the
 * number of cells (may exceed cap, in which case only cap are written). */
int64_t or_traverse_cells(const int64_t A[3], const int64_t B[3], int64_t* out, int64_t cap)
{
    or_collect ctx = {out, cap, 0};
    or_traverse(A, B, collect_visit, &ctx);
    return ctx.n;
}

typedef struct {
    const or_params* p;
    uint32_t* passes;
    int64_t end[3];
    int64_t visits;
} pass_ctx;

/* Sec. III-A: misses are rays that pass through a voxel but do not end in
 * it. Every in-window cell of the traversal other than the endpoint cell is
 * counted (the sensor's own cell included). */
static void pass_visit(void* vctx, const int64_t cell[3])
{
    pass_ctx* ctx = (pass_ctx*)vctx;
    if (cell[0] == ctx->end[0] && cell[1] == ctx->end[1] && cell[2] == ctx->end[2]) return;
    if (!in_window(ctx->p, cell)) return;
    ctx->passes[lin(ctx->p, cell[0], cell[1], cell[2])] += 1;
    ctx->visits += 1;
}

/* Quantise a map-frame coordinate to 1/256 voxel relative to the origin.
 * Returns 0 if it is beyond the representable range. Reading: endpoints at
 * 1/256 voxel, q = round-half-even(256 (w/res - O)), evaluated as one fused
 * multiply-add s = fma(w, S, -256 O) with S = 256 * (1/res) (both scalings
 * by 256 are exact). */
static int quantise(double w, double S, int64_t origin, int64_t* q)
{
    const double s = fma(w, S, -256.0 * (double)origin);
    if (!(fabs(s) < (double)OR_QLIM)) return 0;
    *q = llrint(s);
    return 1;
}

/* Per-scan update (Sec. III-C pointcloud processing, combined per Sec. III-D).
 *
 * 1. Transform (Sec. III-C): w = R p + t with T = [R | t] row-major 3x4,
 *    w_i = fma(T_i2, pz, fma(T_i1, py, fma(T_i0, px, T_i3))) in FP64 (each
 *    fused multiply-add rounded once, in this order).
 *    The sensor origin is o = (T_03, T_13, T_23).
 * 2. Filter (reading): keep a point iff its components are finite and
 *    0 < r2 <= max_range^2 in the sensor frame, with
 *    r2 = fma(pz, pz, fma(py, py, px * px)) in FP64.
 * 3. Quantise sensor and endpoint (reading, above).
 * 4. Hits and lowest return (Sec. III-A): the endpoint cell, if in the
 *    window, gains one hit and min height min(minz, (float) w_z).
 * 5. Misses (Sec. III-A): every other in-window cell of the traversal gains
 *    one pass.
 * Adding one scan's counts to the resident map and taking the min of the
 * heights is the combination rule of Sec. III-D (hits and misses add, min
 * heights take the minimum), so accumulating scan after scan into one map
 * equals combining the per-scan maps.
 * Parity: hits pinned (sum of hits equals in-window valid points, brute
 * force binning); passes pinned through the traversal pin plus per-ray
 * count identities; the transform is pinned by identity and exact
 * permutation poses. */
void or_ingest(const or_params* p, const int64_t origin[3], uint32_t* hits, uint32_t* passes,
               float* minz, const float* pts, int64_t n, int32_t stride, const double T[12],
               or_stats* st)
{
    const double S = 256.0 * (1.0 / p->res);
    const double r2max = p->max_range * p->max_range;
    int64_t qo[3];
    int sensor_ok = 1;
    for (int a = 0; a < 3; ++a)
        if (!quantise(T[4 * a + 3], S, origin[a], &qo[a])) sensor_ok = 0;

    for (int64_t i = 0; i < n; ++i) {
        st->points_in += 1;
        const float fx = pts[i * stride + 0], fy = pts[i * stride + 1], fz = pts[i * stride + 2];
        if (!isfinite(fx) || !isfinite(fy) || !isfinite(fz)) continue;
        const double px = (double)fx, py = (double)fy, pz = (double)fz;
        const double r2 = fma(pz, pz, fma(py, py, px * px));
        if (!(r2 > 0.0 && r2 <= r2max)) continue;
        if (!sensor_ok) continue;
        double w[3];
        for (int a = 0; a < 3; ++a)
            w[a] = fma(T[4 * a + 2], pz, fma(T[4 * a + 1], py, fma(T[4 * a + 0], px, T[4 * a + 3])));
        int64_t q[3];
        int ok = 1;
        for (int a = 0; a < 3; ++a)
            if (!quantise(w[a], S, origin[a], &q[a])) ok = 0;
        if (!ok) continue;
        st->rays_valid += 1;

        int64_t ce[3];
        for (int a = 0; a < 3; ++a) ce[a] = floor_div(q[a], 256);
        if (in_window(p, ce)) {
            const int64_t k = lin(p, ce[0], ce[1], ce[2]);
            hits[k] += 1;
            const float wz = (float)w[2];
            if (wz < minz[k]) minz[k] = wz;
            st->hits_in_window += 1;
        }
        pass_ctx ctx;
        ctx.p = p;
        ctx.passes = passes;
        ctx.end[0] = ce[0];
        ctx.end[1] = ce[1];
        ctx.end[2] = ce[2];
        ctx.visits = 0;
        or_traverse(qo, q, pass_visit, &ctx);
        st->pass_visits += ctx.visits;
    }
}

/* ---------------------------------------------------------------------- */
/* 2D products (Sec. III-D). */

/* Height (Sec. III-D): the lowest return of the lowest occupied voxel of
 * each column, i.e. the minimum of minz over the occupied voxels of the
 * column; NaN where the column has no occupied voxel.
 * Positive obstacles (Sec. III-D), reading: K = occupied voxels of the
 * column whose lowest return lies in [h + obs_min_h, h + obs_max_h];
 * obstacle iff K is not empty; density = H / (H + M) with H, M the sums of
 * hits and passes over K, which is the mean of the per-voxel opacity
 * hits / (hits + passes) weighted by the rays each voxel saw; hard iff
 * H * hard_den >= hard_num * (H + M), soft otherwise. density is 0 where
 * there is no obstacle.
 * flags: bit0 obstacle, bit1 hard, bit2 soft (bit3 set by or_negative). */
void or_columns(const or_params* p, const uint32_t* hits, const uint32_t* passes,
                const float* minz, float* height, float* density, uint8_t* flags)
{
    for (int64_t ix = 0; ix < p->nx; ++ix)
        for (int64_t iy = 0; iy < p->ny; ++iy) {
            const int64_t px = ix * p->ny + iy;
            float h = NAN;
            int have = 0;
            for (int64_t iz = 0; iz < p->nz; ++iz) {
                const int64_t k = lin(p, ix, iy, iz);
                if (hits[k] >= 1) {
                    if (!have || minz[k] < h) h = minz[k];
                    have = 1;
                }
            }
            height[px] = h;
            uint64_t H = 0, M = 0;
            int obstacle = 0;
            if (have) {
                for (int64_t iz = 0; iz < p->nz; ++iz) {
                    const int64_t k = lin(p, ix, iy, iz);
                    if (hits[k] < 1) continue;
                    const double above = (double)minz[k] - (double)h;
                    if ((double)p->obs_min_h <= above && above <= (double)p->obs_max_h) {
                        obstacle = 1;
                        H += hits[k];
                        M += passes[k];
                    }
                }
            }
            uint8_t f = 0;
            density[px] = 0.0f;
            if (obstacle) {
                density[px] = (float)((double)H / (double)(H + M));
                const int hard = H * (uint64_t)p->hard_den >= (uint64_t)p->hard_num * (H + M);
                f |= 1u;
                f |= hard ? 2u : 4u;
            }
            flags[px] = f;
        }
}

/* Slope and roughness (Sec. III-D): least-squares plane over the N x N
 * window of pixels around each pixel; roughness is the mean squared error
 * of that fit. Readings: only defined pixels of the window enter the fit;
 * the centre pixel must be defined; at least slope_min_px pixels and a
 * non-singular normal matrix are needed, else both are NaN. The plane
 * z = a i + b j + c is fitted over integer pixel offsets (i, j) with z the
 * height minus the centre height; slope = atan(hypot(a, b) / res) radians;
 * roughness = (1/n) sum of squared residuals, square metres. The 3x3 normal
 * equations are solved by Cramer's rule in FP64.
 * Pinned by closed forms: a plane tilted by a known angle sampled at pixel
 * centres, a flat plane, and a checkerboard checked against a library
 * least-squares routine. */
void or_slope(const or_params* p, const float* height, float* slope, float* rough)
{
    const int32_t r = p->slope_n / 2;
    for (int64_t ix = 0; ix < p->nx; ++ix)
        for (int64_t iy = 0; iy < p->ny; ++iy) {
            const int64_t px = ix * p->ny + iy;
            slope[px] = NAN;
            rough[px] = NAN;
            const float h0 = height[px];
            if (isnan(h0)) continue;
            /* normal matrix sums (integers) and right-hand side */
            int64_t n = 0, si = 0, sj = 0, sii = 0, sjj = 0, sij = 0;
            double sz = 0.0, siz = 0.0, sjz = 0.0;
            for (int32_t i = -r; i <= r; ++i)
                for (int32_t j = -r; j <= r; ++j) {
                    const int64_t x = ix + i, y = iy + j;
                    if (x < 0 || x >= p->nx || y < 0 || y >= p->ny) continue;
                    const float h = height[x * p->ny + y];
                    if (isnan(h)) continue;
                    const double z = (double)h - (double)h0;
                    n += 1;
                    si += i;
                    sj += j;
                    sii += (int64_t)i * i;
                    sjj += (int64_t)j * j;
                    sij += (int64_t)i * j;
                    sz += z;
                    siz += (double)i * z;
                    sjz += (double)j * z;
                }
            if (n < p->slope_min_px) continue;
            /* [sii sij si; sij sjj sj; si sj n] [a b c]^T = [siz sjz sz]^T */
            const int64_t det = sii * (sjj * n - sj * sj) - sij * (sij * n - sj * si) +
                                si * (sij * sj - sjj * si);
            if (det == 0) continue;
            const double D = (double)det;
            const double da = siz * (double)(sjj * n - sj * sj) - (double)sij * (sjz * (double)n - (double)sj * sz) +
                              (double)si * (sjz * (double)sj - (double)sjj * sz);
            const double db = (double)sii * (sjz * (double)n - (double)sj * sz) - siz * (double)(sij * n - sj * si) +
                              (double)si * ((double)sij * sz - sjz * (double)si);
            const double dc = (double)sii * ((double)sjj * sz - (double)sj * sjz) -
                              (double)sij * ((double)sij * sz - (double)si * sjz) +
                              siz * (double)(sij * sj - sjj * si);
            const double a = da / D, b = db / D, c = dc / D;
            double sse = 0.0;
            for (int32_t i = -r; i <= r; ++i)
                for (int32_t j = -r; j <= r; ++j) {
                    const int64_t x = ix + i, y = iy + j;
                    if (x < 0 || x >= p->nx || y < 0 || y >= p->ny) continue;
                    const float h = height[x * p->ny + y];
                    if (isnan(h)) continue;
                    const double z = (double)h - (double)h0;
                    const double e = z - (a * i + b * j + c);
                    sse += e * e;
                }
            slope[px] = (float)atan(hypot(a, b) / p->res);
            rough[px] = (float)(sse / (double)n);
        }
}

/* Negative obstacles (Sec. III-D, Fig. 3 and Fig. 4). Only pixels whose
 * height is undefined are tested. From the pixel, four cones are searched
 * outwards ring by ring (Chebyshev distance d = 1 .. neg_max_px):
 *   +x: cells (x+d, y+j), |j| <= d     -x: cells (x-d, y+j), |j| <= d
 *   +y: cells (x+i, y+d), |i| <= d     -y: cells (x+i, y-d), |i| <= d
 * A cone stops at the first ring holding at least one defined in-grid
 * pixel, and takes the lowest height on that ring as its assumed height; it
 * stops without a height when its ring lies outside the grid or d passes
 * neg_max_px. Readings: four cones (the four colours of Fig. 4), the lowest
 * height of the ring as the cone's value, at least two heights needed. The
 * pixel is a negative obstacle iff the largest difference between the found
 * heights, max - min, exceeds neg_thresh (strictly). Sets bit3 of flags.
 * Pinned by the Fig. 4 scenario (three cones find ground, one reaches the
 * grid edge) and by hole grids with a known Delta H. */
void or_negative(const or_params* p, const float* height, uint8_t* flags)
{
    static const int dirs[4][2] = {{+1, 0}, {-1, 0}, {0, +1}, {0, -1}};
    for (int64_t ix = 0; ix < p->nx; ++ix)
        for (int64_t iy = 0; iy < p->ny; ++iy) {
            const int64_t px = ix * p->ny + iy;
            if (!isnan(height[px])) continue;
            int nfound = 0;
            float lo = 0.0f, hi = 0.0f;
            for (int c = 0; c < 4; ++c) {
                for (int32_t d = 1; d <= p->neg_max_px; ++d) {
                    /* the ring's fixed coordinate along the cone's axis */
                    int64_t fx = ix + (int64_t)dirs[c][0] * d, fy = iy + (int64_t)dirs[c][1] * d;
                    const int along_x = dirs[c][0] != 0;
                    if (along_x ? (fx < 0 || fx >= p->nx) : (fy < 0 || fy >= p->ny)) break;
                    int found = 0;
                    float best = 0.0f;
                    for (int32_t s = -d; s <= d; ++s) {
                        const int64_t x = along_x ? fx : ix + s;
                        const int64_t y = along_x ? iy + s : fy;
                        if (x < 0 || x >= p->nx || y < 0 || y >= p->ny) continue;
                        const float h = height[x * p->ny + y];
                        if (isnan(h)) continue;
                        if (!found || h < best) best = h;
                        found = 1;
                    }
                    if (found) {
                        if (nfound == 0 || best < lo) lo = best;
                        if (nfound == 0 || best > hi) hi = best;
                        nfound += 1;
                        break;
                    }
                }
            }
            if (nfound >= 2 && ((double)hi - (double)lo) > (double)p->neg_thresh)
                flags[px] |= 8u;
        }
}

/* All 2D products in the order of Sec. III-D. */
void or_extract(const or_params* p, const uint32_t* hits, const uint32_t* passes, const float* minz,
                float* height, float* density, uint8_t* flags, float* slope, float* rough)
{
    or_columns(p, hits, passes, minz, height, density, flags);
    or_slope(p, height, slope, rough);
    or_negative(p, height, flags);
}

/* Lookup-table encoding of the map (Sec. III-A): the data array holds the
 * metrics (hits, misses, lowest return) of the occupied voxels, in the
 * order of their logical linear index; the lookup table, one entry per
 * voxel, holds an occupied voxel's index in the data array and
 * -1 - N_m (N_m = the voxel's misses) for every other voxel. Entries are
 * int64 so that -1 - N_m is exact for any 32-bit miss count. Data entries
 * at or beyond `cap` are not written. Returns the number of occupied
 * voxels. Pinned by tests: decoding the table gives the state back, the
 * indices rise with the linear index, and a hand-built grid. */
int64_t or_lut(const or_params* p, const uint32_t* hits, const uint32_t* passes, const float* minz, int64_t* lut,
               uint32_t* d_hits, uint32_t* d_passes, float* d_minz, int64_t cap)
{
    const int64_t V = (int64_t)p->nx * p->ny * p->nz;
    int64_t k = 0;
    for (int64_t i = 0; i < V; ++i) {
        if (hits[i] >= 1) {
            lut[i] = k;
            if (k < cap) {
                d_hits[k] = hits[i];
                d_passes[k] = passes[i];
                d_minz[k] = minz[i];
            }
            k += 1;
        } else {
            lut[i] = -1 - (int64_t)passes[i];
        }
    }
    return k;
}
