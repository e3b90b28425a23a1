/*
 * Pointer-octree oracle for "Background Modeling Using Octree Color
 * Quantization" (arXiv 1412.1945).
 *
 * TEST INFRASTRUCTURE.  This file is the plain, slow, obviously-correct CPU
 * statement of what the method computes.  Only the test suite, the smoke check
 * and the benchmark's CPU-baseline / reference arm may load it; the product path
 * (the CUDA library) never calls it and shares no code with it.
 *
 * It follows the paper's own data structure and procedures:
 *   - an octree node has eight children (Sec. 2);
 *   - Store Color (Alg. 1) inserts a colour by walking one bit of red, green
 *     and blue per level, most significant bit first, creating missing
 *     children; stopping the walk after `depth` levels is the paper's pruning
 *     of dropping the bottom levels (Sec. 2), so a leaf at depth d keeps
 *     the d most significant bits of each channel;
 *   - one tree is built per training frame and per region (Sec. 3, Sec. 4);
 *   - Merge Trees (Alg. 2) keeps child i of a merged node when at least
 *     T of the N trees have child i there, then recurses into kept children;
 *   - Check Color (Alg. 3) walks the merged tree; a missing child (or an empty
 *     tree) means the colour is not background, i.e. foreground.
 *
 * Readings of points the paper leaves open (each also listed in the design notes):
 *   R1  child index = (red bit << 2) | (green bit << 1) | blue bit; the
 *       printed sum of the three bits is read as bit concatenation, since
 *       eight children need three bits.
 *   R2  the loop from the most significant bit to the number of levels walks
 *       bits 7, 6, ..., 8-d: d levels.
 *   R3  the threshold test on the fraction of trees holding a child is taken
 *       with an integer count threshold T (keep iff count >= T); a fraction t
 *       maps to T = ceil(t * N).
 *   R6  Merge Trees recurses on the child arrays with the level increased by
 *       one, stops at depth d, and a NULL tree does not count.
 *   R8  only depth-d nodes are colours: an internal merged node with no kept
 *       child below it does not make a colour background.
 *   R9  a region with an empty merged tree classifies every pixel foreground.
 *   R11 regions: whole frame (kind 0) is one region; b x b blocks (kind 1) are
 *       numbered row-major, (y/b)*ceil(W/b) + x/b, with partial edge blocks;
 *       single pixels (kind 2) are numbered y*W + x.
 *   R12 the mask is u8 with 1 = foreground, 0 = background.
 *
 * Pins (tests/test_oracle_pins.py, tests/test_oracle_next.py): every function
 * here is checked against closed forms, invariants, hand-derived cases or the
 * set-based restatement.  Parity unpinned (conventions the paper does not fix,
 * so nothing it prints can confirm them): the bit order R1 inside exported
 * path codes (classification does not depend on it), the fraction-to-T
 * rounding R3, and the serving window semantics built on these functions.
 *
 * A leaf's identity ("path code") is the sequence of child indices from the
 * root: code = sum over levels l of index_l * 8^(d-1-l).  The merged model of a
 * region is exported as a bitset of 8^d bits in u64 words, leaf c at bit c%64
 * of word c/64 (one word when d <= 2).
 *
 * Frames are HWC RGB8, no row padding: pixel (f, y, x) channel ch at
 * ((f*H + y)*W + x)*3 + ch.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct octree_node {
  struct octree_node *child[8];
  uint64_t count; /* pixels whose walk ended at this node (leaf pixel counter) */
  uint32_t code;  /* path code, filled in by label_leaves() */
} octree_node;

static octree_node *create_node(void) { return (octree_node *)calloc(1, sizeof(octree_node)); }

static void free_tree(octree_node *n) {
  if (!n) return;
  for (int i = 0; i < 8; ++i) free_tree(n->child[i]);
  free(n);
}

/* Child index at bit i of a colour (R1). */
static int child_index(uint8_t r, uint8_t g, uint8_t b, int i) {
  return (((r >> i) & 1) << 2) | (((g >> i) & 1) << 1) | ((b >> i) & 1);
}

/* Store Color, Alg. 1: returns the (possibly new) root, or NULL when a node
 * cannot be allocated. */
static octree_node *store_color(octree_node *root, uint8_t r, uint8_t g, uint8_t b, int levels) {
  if (root == NULL) {
    root = create_node();
    if (!root) return NULL;
  }
  octree_node *temp = root;
  for (int i = 7; i >= 8 - levels; --i) { /* MSB down to the pruning height (R2) */
    int index = child_index(r, g, b, i);
    if (temp->child[index] != NULL) {
      temp = temp->child[index];
    } else {
      temp->child[index] = create_node();
      if (!temp->child[index]) return NULL;
      temp = temp->child[index];
    }
  }
  temp->count++;
  return root;
}

/* Merge Trees, Alg. 2 (with reading R6): merges the n trees whose roots are
 * given (entries may be NULL) into a new tree and returns its root. */
static octree_node *merge_trees(octree_node *const *roots, int n, int threshold, int level, int levels,
                                int *oom) {
  octree_node *result = create_node();
  if (!result) {
    *oom = 1;
    return NULL;
  }
  if (level == levels) return result; /* reached the pruning height: a leaf */
  int keep[8];
  for (int i = 0; i < 8; ++i) {
    int count = 0;
    for (int j = 0; j < n; ++j)
      if (roots[j] != NULL && roots[j]->child[i] != NULL) count++;
    keep[i] = count >= threshold; /* R3 */
  }
  octree_node **temp_root = (octree_node **)malloc(sizeof(octree_node *) * (size_t)(n > 0 ? n : 1));
  if (!temp_root) {
    *oom = 1;
    return result;
  }
  for (int i = 0; i < 8; ++i) {
    if (!keep[i]) continue;
    for (int j = 0; j < n; ++j) temp_root[j] = roots[j] ? roots[j]->child[i] : NULL;
    result->child[i] = merge_trees(temp_root, n, threshold, level + 1, levels, oom);
    if (*oom) break;
  }
  free(temp_root);
  return result;
}

/* Check Color, Alg. 3: 1 when the colour's path exists down to the pruning
 * height (background), 0 otherwise (R8, R9). */
static int check_color(const octree_node *root, uint8_t r, uint8_t g, uint8_t b, int levels) {
  if (root == NULL) return 0;
  const octree_node *temp = root;
  for (int i = 7; i >= 8 - levels; --i) {
    int index = child_index(r, g, b, i);
    if (temp->child[index] != NULL)
      temp = temp->child[index];
    else
      return 0;
  }
  return 1;
}

/* ---- leaf paths <-> bitsets -------------------------------------------- */

static int64_t words_per_region(int depth) { return depth <= 2 ? 1 : (int64_t)1 << (3 * depth - 6); }

static void export_leaves(const octree_node *n, int level, int levels, uint64_t code, uint64_t *words) {
  if (level == levels) {
    words[code >> 6] |= (uint64_t)1 << (code & 63);
    return;
  }
  for (int i = 0; i < 8; ++i)
    if (n->child[i]) export_leaves(n->child[i], level + 1, levels, code * 8 + (uint64_t)i, words);
}

/* Rebuilds a tree whose depth-d leaves are exactly the set bits of `words`. */
static octree_node *import_leaves(const uint64_t *words, int levels, int *oom) {
  octree_node *root = create_node();
  if (!root) {
    *oom = 1;
    return NULL;
  }
  const uint64_t nleaves = (uint64_t)1 << (3 * levels);
  for (uint64_t c = 0; c < nleaves; ++c) {
    if (!((words[c >> 6] >> (c & 63)) & 1)) continue;
    octree_node *temp = root;
    for (int l = 0; l < levels; ++l) {
      int index = (int)((c >> (3 * (levels - 1 - l))) & 7);
      if (!temp->child[index]) {
        temp->child[index] = create_node();
        if (!temp->child[index]) {
          *oom = 1;
          return root;
        }
      }
      temp = temp->child[index];
    }
  }
  return root;
}

static void tree_stats(const octree_node *n, int level, int levels, int64_t *leaves, int64_t *sum, int64_t *nodes) {
  (*nodes)++;
  if (level == levels) {
    (*leaves)++;
    *sum += (int64_t)n->count;
    return;
  }
  for (int i = 0; i < 8; ++i)
    if (n->child[i]) tree_stats(n->child[i], level + 1, levels, leaves, sum, nodes);
}

/* ---- regions (R11) ------------------------------------------------------ */

int64_t oracle_region_count(int H, int W, int kind, int block) {
  if (H < 1 || W < 1) return -1;
  if (kind == 0) return 1;
  if (kind == 1) {
    if (block < 1) return -1;
    return (int64_t)((H + block - 1) / block) * ((W + block - 1) / block);
  }
  if (kind == 2) return (int64_t)H * W;
  return -1;
}

static void region_rect(int H, int W, int kind, int block, int64_t r, int *y0, int *y1, int *x0, int *x1) {
  if (kind == 0) {
    *y0 = 0, *y1 = H, *x0 = 0, *x1 = W;
  } else if (kind == 1) {
    int bw = (W + block - 1) / block;
    int by = (int)(r / bw), bx = (int)(r % bw);
    *y0 = by * block;
    *x0 = bx * block;
    *y1 = *y0 + block < H ? *y0 + block : H;
    *x1 = *x0 + block < W ? *x0 + block : W;
  } else {
    *y0 = (int)(r / W);
    *x0 = (int)(r % W);
    *y1 = *y0 + 1;
    *x1 = *x0 + 1;
  }
}

static int check_args(int H, int W, int kind, int block, int depth) {
  if (oracle_region_count(H, W, kind, block) < 1) return 1;
  if (depth < 1 || depth > 8) return 1;
  return 0;
}

/* Number of trees when one tree holds `group` consecutive frames (Sec. 3
 * allows one tree per frame or per group of frames); the last group holds the
 * remaining frames. */
static int tree_count(int N, int group) { return (N + group - 1) / group; }

/* Builds the trees of region r: tree j holds the region's pixels of training
 * frames [j*group, j*group + group) (Store Color over each pixel); group = 1
 * gives one tree per frame. */
static int build_region_trees(const uint8_t *frames, int N, int group, int H, int W, int kind, int block,
                              int depth, int64_t r, octree_node **roots) {
  int y0, y1, x0, x1;
  region_rect(H, W, kind, block, r, &y0, &y1, &x0, &x1);
  for (int j = 0; j < tree_count(N, group); ++j) roots[j] = NULL;
  for (int f = 0; f < N; ++f) {
    octree_node **root = &roots[f / group];
    for (int y = y0; y < y1; ++y)
      for (int x = x0; x < x1; ++x) {
        const uint8_t *p = frames + (((size_t)f * H + y) * W + x) * 3;
        octree_node *nr = store_color(*root, p[0], p[1], p[2], depth);
        if (!nr) return 1;
        *root = nr;
      }
  }
  return 0;
}

/* Classifies the region's pixels of F frames against `tree`; writes masks either
 * at their frame positions (gathered == 0) or consecutively from *cursor. */
static void classify_region(const octree_node *tree, const uint8_t *frames, int F, int H, int W, int kind,
                            int block, int depth, int64_t r, uint8_t *mask, int gathered, size_t *cursor) {
  int y0, y1, x0, x1;
  region_rect(H, W, kind, block, r, &y0, &y1, &x0, &x1);
  for (int f = 0; f < F; ++f)
    for (int y = y0; y < y1; ++y)
      for (int x = x0; x < x1; ++x) {
        size_t pix = ((size_t)f * H + y) * W + x;
        const uint8_t *p = frames + pix * 3;
        uint8_t fg = check_color(tree, p[0], p[1], p[2], depth) ? 0 : 1;
        if (gathered)
          mask[(*cursor)++] = fg;
        else
          mask[pix] = fg;
      }
}

/*
 * Build (Sec. 3, Alg. 1 + Alg. 2) and, when test frames are given, classify
 * (Sec. 4, Alg. 3) region by region, so only one region's trees are alive.
 *
 * train: N frames; test: F frames (may be NULL with F = 0).
 * regions: ids to process (NULL = all, in order); nreg: their number.
 * model_out: one row of words_per_region(depth) u64 per processed region (may be NULL).
 * mask_out: F*H*W bytes when regions == NULL; otherwise gathered, for each
 *   listed region, each frame, its pixels in row-major order (may be NULL).
 * Returns 0 on success, 1 on bad arguments, 2 on allocation failure.
 */
/*
 * As oracle_run, with one tree per group of `group` consecutive training
 * frames (Sec. 3); T counts groups, 1 <= T <= ceil(N / group).
 */
int oracle_run_groups(const uint8_t *train, int N, int group, const uint8_t *test, int F, int H, int W, int kind,
                      int block, int depth, int T, const int64_t *regions, int64_t nreg, uint64_t *model_out,
                      uint8_t *mask_out) {
  if (check_args(H, W, kind, block, depth) || N < 1 || group < 1 || T < 1 || T > tree_count(N, group) || F < 0 ||
      !train)
    return 1;
  const int G = tree_count(N, group);
  const int64_t R = oracle_region_count(H, W, kind, block);
  const int64_t nr = regions ? nreg : R;
  const int64_t wpr = words_per_region(depth);
  octree_node **roots = (octree_node **)malloc(sizeof(octree_node *) * (size_t)G);
  if (!roots) return 2;
  size_t cursor = 0;
  int rc = 0;
  for (int64_t k = 0; k < nr && rc == 0; ++k) {
    const int64_t r = regions ? regions[k] : k;
    if (r < 0 || r >= R) {
      rc = 1;
      break;
    }
    if (build_region_trees(train, N, group, H, W, kind, block, depth, r, roots)) rc = 2;
    int oom = 0;
    octree_node *merged = rc ? NULL : merge_trees(roots, G, T, 0, depth, &oom);
    if (oom) rc = 2;
    for (int j = 0; j < G; ++j) free_tree(roots[j]);
    if (rc == 0 && model_out) {
      uint64_t *row = model_out + (size_t)k * (size_t)wpr;
      memset(row, 0, sizeof(uint64_t) * (size_t)wpr);
      export_leaves(merged, 0, depth, 0, row);
    }
    if (rc == 0 && mask_out && test && F > 0)
      classify_region(merged, test, F, H, W, kind, block, depth, r, mask_out, regions != NULL, &cursor);
    free_tree(merged);
  }
  free(roots);
  return rc;
}

/* One tree per training frame (Sec. 3, the hot path's case). */
int oracle_run(const uint8_t *train, int N, const uint8_t *test, int F, int H, int W, int kind, int block,
               int depth, int T, const int64_t *regions, int64_t nreg, uint64_t *model_out, uint8_t *mask_out) {
  return oracle_run_groups(train, N, 1, test, F, H, W, kind, block, depth, T, regions, nreg, model_out, mask_out);
}

/* Build only: oracle_run without test frames. */
int oracle_build(const uint8_t *train, int N, int H, int W, int kind, int block, int depth, int T,
                 const int64_t *regions, int64_t nreg, uint64_t *model_out) {
  return oracle_run(train, N, NULL, 0, H, W, kind, block, depth, T, regions, nreg, model_out, NULL);
}

/*
 * Classify against an exported model: each region's bitset row is turned back
 * into a pointer tree and Check Color (Alg. 3) runs on it.  model rows follow
 * `regions` (or all regions in order); mask_out layout as in oracle_run.
 */
int oracle_classify(const uint64_t *model, int H, int W, int kind, int block, int depth, const uint8_t *frames,
                    int F, const int64_t *regions, int64_t nreg, uint8_t *mask_out) {
  if (check_args(H, W, kind, block, depth) || F < 0 || !model || !mask_out || (F > 0 && !frames)) return 1;
  const int64_t R = oracle_region_count(H, W, kind, block);
  const int64_t nr = regions ? nreg : R;
  const int64_t wpr = words_per_region(depth);
  size_t cursor = 0;
  for (int64_t k = 0; k < nr; ++k) {
    const int64_t r = regions ? regions[k] : k;
    if (r < 0 || r >= R) return 1;
    int oom = 0;
    octree_node *tree = import_leaves(model + (size_t)k * (size_t)wpr, depth, &oom);
    if (oom) {
      free_tree(tree);
      return 2;
    }
    classify_region(tree, frames, F, H, W, kind, block, depth, r, mask_out, regions != NULL, &cursor);
    free_tree(tree);
  }
  return 0;
}

/*
 * Statistics of the pruned per-frame trees of one frame, per region: number of
 * depth-d leaves, sum of the leaf pixel counters, and number of nodes (root
 * included).  Used to pin the oracle (counts must sum to the region's pixels).
 */
int oracle_tree_stats(const uint8_t *frame, int H, int W, int kind, int block, int depth, int64_t *leaves_out,
                      int64_t *count_sum_out, int64_t *nodes_out) {
  if (check_args(H, W, kind, block, depth) || !frame) return 1;
  const int64_t R = oracle_region_count(H, W, kind, block);
  for (int64_t r = 0; r < R; ++r) {
    octree_node *root = NULL;
    if (build_region_trees(frame, 1, 1, H, W, kind, block, depth, r, &root)) {
      free_tree(root);
      return 2;
    }
    int64_t leaves = 0, sum = 0, nodes = 0;
    if (root) tree_stats(root, 0, depth, &leaves, &sum, &nodes);
    if (leaves_out) leaves_out[r] = leaves;
    if (count_sum_out) count_sum_out[r] = sum;
    if (nodes_out) nodes_out[r] = nodes;
    free_tree(root);
  }
  return 0;
}

static void label_leaves(octree_node *n, int level, int levels, uint32_t code) {
  if (level == levels) {
    n->code = code;
    return;
  }
  for (int i = 0; i < 8; ++i)
    if (n->child[i]) label_leaves(n->child[i], level + 1, levels, code * 8u + (uint32_t)i);
}

/*
 * Path codes of n colours (rgb: n x 3 bytes): all colours go into one tree with
 * Store Color, each leaf is labelled with its path from the root, and each
 * colour is then walked to its leaf to read the label.
 */
int oracle_leaf_codes(const uint8_t *rgb, int64_t n, int depth, uint32_t *codes_out) {
  if (depth < 1 || depth > 8 || n < 0 || (n > 0 && (!rgb || !codes_out))) return 1;
  octree_node *root = NULL;
  for (int64_t k = 0; k < n; ++k) {
    root = store_color(root, rgb[3 * k], rgb[3 * k + 1], rgb[3 * k + 2], depth);
    if (!root) return 2;
  }
  if (!root) return 0;
  label_leaves(root, 0, depth, 0);
  for (int64_t k = 0; k < n; ++k) {
    const octree_node *t = root;
    for (int i = 7; i >= 8 - depth; --i) t = t->child[child_index(rgb[3 * k], rgb[3 * k + 1], rgb[3 * k + 2], i)];
    codes_out[k] = t->code;
  }
  free_tree(root);
  return 0;
}

int64_t oracle_words_per_region(int depth) { return (depth < 1 || depth > 8) ? -1 : words_per_region(depth); }

/*
 * Redraw (Sec. 2, Fig. 2): each colour is stored in a tree pruned at `depth`
 * levels, and the newly exposed leaf gives the colour back with the depth
 * original bits of each channel and zeros below.  The leaf's bits are read off
 * its path: level l's child index carries bit 7 - l of red, green and blue.
 */
int oracle_redraw(const uint8_t *rgb, int64_t n, int depth, uint8_t *out) {
  if (depth < 1 || depth > 8 || n < 0 || (n > 0 && (!rgb || !out))) return 1;
  for (int64_t k = 0; k < n; ++k) {
    const uint8_t r = rgb[3 * k], g = rgb[3 * k + 1], b = rgb[3 * k + 2];
    uint8_t lr = 0, lg = 0, lb = 0;
    for (int i = 7; i >= 8 - depth; --i) {
      const int index = child_index(r, g, b, i);
      lr |= (uint8_t)(((index >> 2) & 1) << i);
      lg |= (uint8_t)(((index >> 1) & 1) << i);
      lb |= (uint8_t)((index & 1) << i);
    }
    out[3 * k] = lr, out[3 * k + 1] = lg, out[3 * k + 2] = lb;
  }
  return 0;
}

/*
 * Confusion counts of a foreground mask against ground truth, per frame
 * (Sec. 5: true/false positives and negatives; foreground = positive, a
 * non-zero byte is foreground in both).  counts_out: F rows of
 * {Tp, Fp, Tn, Fn}.
 */
int oracle_confusion(const uint8_t *mask, const uint8_t *gt, int64_t F, int64_t npix, uint64_t *counts_out) {
  if (F < 0 || npix < 0 || !counts_out || (F > 0 && npix > 0 && (!mask || !gt))) return 1;
  for (int64_t f = 0; f < F; ++f) {
    uint64_t tp = 0, fp = 0, tn = 0, fn = 0;
    for (int64_t p = 0; p < npix; ++p) {
      const int predicted = mask[f * npix + p] != 0, actual = gt[f * npix + p] != 0;
      if (predicted && actual) ++tp;
      else if (predicted && !actual) ++fp;
      else if (!predicted && !actual) ++tn;
      else ++fn;
    }
    counts_out[4 * f] = tp, counts_out[4 * f + 1] = fp, counts_out[4 * f + 2] = tn, counts_out[4 * f + 3] = fn;
  }
  return 0;
}
