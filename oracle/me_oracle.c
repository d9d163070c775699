/*
 * CPU oracle for edge detection of binary images by the method of masks.
 *
 * TEST INFRASTRUCTURE ONLY.  The test suite, the smoke check and the
 * benchmark's CPU-baseline leg are the only callers allowed to load this
 * library.  It shares no code, header or constant with the CUDA library.
 *
 * Storage: one byte per pixel, row-major u8[h][w]; 0 = black, 1 = white
 * (Section 2: the colour data of a monochrome image is one bit per pixel,
 * 0 for black and 1 for white).  Any non-zero byte is read as white.
 *
 * Neighbours are numbered as in Fig. 1:      3 2 1
 *                                            4 P 8
 *                                            5 6 7
 * so 2 is the pixel above P, 4 the one to its left, 6 the one below and 8
 * the one to its right.  A neighbour outside the image takes the boundary
 * colour: boundary 0 means outside pixels are white, boundary 1 black.
 *
 * Every function returns 0 on success and -1 on a bad argument.
 */
#include <stddef.h>
#include <stdint.h>

/* Colour of pixel (x, y) as 0 (black) or 1 (white); outside -> outside. */
static int pixel(const uint8_t *img, int w, int h, int x, int y, int outside)
{
    if (x < 0 || y < 0 || x >= w || y >= h)
        return outside;
    return img[(size_t)y * (size_t)w + (size_t)x] != 0;
}

static int outside_colour(int boundary)
{
    return boundary ? 0 : 1;
}

static int bad_args(const void *img, int w, int h, int boundary)
{
    return img == NULL || w < 0 || h < 0 || (boundary != 0 && boundary != 1);
}

/*
 * Section 3: the mask is the negative image, every pixel inverted.
 * out[y][x] = 1 where the image is black.
 */
int me_oracle_mask(const uint8_t *img, int w, int h, uint8_t *out)
{
    if (bad_args(img, w, h, 0) || out == NULL)
        return -1;
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x)
            out[(size_t)y * w + x] = pixel(img, w, h, x, y, 1) ? 0 : 1;
    return 0;
}

/*
 * Section 1, the Boolean function Edge(p) = (p)' and (2 or 4 or 6 or 8),
 * evaluated pixel by pixel the way the traditional scan of Section 1 does:
 * a black pixel with at least one white 4-neighbour is an edge point.
 * out[y][x] = 1 for an edge point, 0 otherwise.
 */
int me_oracle_edges(const uint8_t *img, int w, int h, int boundary, uint8_t *out)
{
    if (bad_args(img, w, h, boundary) || out == NULL)
        return -1;
    const int o = outside_colour(boundary);
    for (int y = 0; y < h; ++y) {
        for (int x = 0; x < w; ++x) {
            int p  = pixel(img, w, h, x, y, o);
            int n2 = pixel(img, w, h, x, y - 1, o);
            int n4 = pixel(img, w, h, x - 1, y, o);
            int n6 = pixel(img, w, h, x, y + 1, o);
            int n8 = pixel(img, w, h, x + 1, y, o);
            out[(size_t)y * w + x] = (uint8_t)(!p && (n2 || n4 || n6 || n8));
        }
    }
    return 0;
}

/* me_oracle_edges over `count` images of the same size stored back to back. */
int me_oracle_edges_many(const uint8_t *imgs, int count, int w, int h,
                         int boundary, uint8_t *out)
{
    if (count < 0 || imgs == NULL || out == NULL)
        return -1;
    size_t n = (size_t)w * (size_t)h;
    for (int i = 0; i < count; ++i)
        if (me_oracle_edges(imgs + i * n, w, h, boundary, out + i * n))
            return -1;
    return 0;
}

/*
 * Section 4: the four fundamental edges.  Each is the mask ANDed with the
 * image moved one pixel.  For the left edge the image is moved one pixel to
 * the right, so the mask pixel at (x, y) meets the image pixel at (x-1, y):
 *     left  = black P with a white neighbour 4  (Fig. 2 b)
 *     right = black P with a white neighbour 8  (Fig. 2 a)
 *     up    = black P with a white neighbour 2  (Fig. 2 c)
 *     down  = black P with a white neighbour 6  (Fig. 2 d)
 * Any output pointer may be NULL to skip that edge.
 */
int me_oracle_fundamental(const uint8_t *img, int w, int h, int boundary,
                          uint8_t *left, uint8_t *right, uint8_t *up,
                          uint8_t *down)
{
    if (bad_args(img, w, h, boundary))
        return -1;
    const int o = outside_colour(boundary);
    for (int y = 0; y < h; ++y) {
        for (int x = 0; x < w; ++x) {
            size_t i = (size_t)y * w + x;
            int m = !pixel(img, w, h, x, y, o);          /* mask pixel */
            if (left)  left[i]  = (uint8_t)(m && pixel(img, w, h, x - 1, y, o));
            if (right) right[i] = (uint8_t)(m && pixel(img, w, h, x + 1, y, o));
            if (up)    up[i]    = (uint8_t)(m && pixel(img, w, h, x, y - 1, o));
            if (down)  down[i]  = (uint8_t)(m && pixel(img, w, h, x, y + 1, o));
        }
    }
    return 0;
}

/*
 * Section 1, second clause of the binary edge-point definition: a black
 * point with at most one black 8-neighbour (an isolated point or the end of
 * a one-pixel line).  out[y][x] = 1 for such a point.
 */
int me_oracle_end_points(const uint8_t *img, int w, int h, int boundary,
                         uint8_t *out)
{
    if (bad_args(img, w, h, boundary) || out == NULL)
        return -1;
    const int o = outside_colour(boundary);
    static const int dx[8] = { 1, 0, -1, -1, -1, 0, 1, 1 };   /* Fig. 1: 1..8 */
    static const int dy[8] = { -1, -1, -1, 0, 1, 1, 1, 0 };
    for (int y = 0; y < h; ++y) {
        for (int x = 0; x < w; ++x) {
            int black_nbrs = 0;
            for (int k = 0; k < 8; ++k)
                black_nbrs += !pixel(img, w, h, x + dx[k], y + dy[k], o);
            int p = pixel(img, w, h, x, y, o);
            out[(size_t)y * w + x] = (uint8_t)(!p && black_nbrs <= 1);
        }
    }
    return 0;
}

/*
 * Thresholding ahead of the method: Section 7 makes a grey photograph
 * binary before finding its edges but names no rule.  Reading taken: one
 * global threshold t, a pixel is white (1) where its grey value is at least
 * t and black (0) below it.  grey is u8[h][pitch], pitch >= w bytes; out is
 * u8[h][w].  t <= 0 makes every pixel white, t > 255 every pixel black.
 */
int me_oracle_threshold(const uint8_t *grey, int w, int h, int pitch, int t, uint8_t *out)
{
    if (grey == NULL || out == NULL || w < 0 || h < 0 || pitch < w)
        return -1;
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x)
            out[(size_t)y * w + x] = (uint8_t)((int)grey[(size_t)y * pitch + x] >= t);
    return 0;
}
