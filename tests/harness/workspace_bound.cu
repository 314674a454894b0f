// Host-only check that deconv_workspace_size covers the layout of every
// launch tuning a plan can be retuned to (the autotuner's candidates, image
// groups, the generic passes, the fused row pass), for several batch
// geometries: compiled against the library's plan.cu and linked with its
// other objects; exit status = number of geometries whose bound is short,
// plus one if some layout puts a bulk-read buffer off a kAlign boundary.
#include "plan.cu"
#include <cstdio>
int main() {
  struct G { const char *name; std::vector<int> M, N; int C, K; };
  std::vector<G> gs = {
    {"c2", {1024}, {1024}, 1, 21}, {"c3", {384,256,384,768,768,768,384,256,512,384,512,512,768,1024,384,1024}, {}, 1, 9},
    {"c4", {1280,1536,512,1536,1536,512,768,1024,512,1536,1280,1280,1024,1024,1024,1024,768,1024,512,1024,1536,1280,1536,512,1280,768,512,512,1536,512,512,1280}, {}, 3, 13},
    {"gen", {96,45,60}, {160,75,54}, 1, 7}, {"rgb", {64,45}, {80,50}, 3, 5}, {"c5", {512,512,512,512,512,512,512,512}, {}, 1, 15},
    {"odd", {100, 75, 243}, {90, 125, 64}, 1, 5}};
  int bad = 0, misaligned = 0;
  for (auto &g : gs) {
    if (g.N.empty()) g.N = g.M;
    deconv_dims d{};
    d.batch = (int)g.M.size(); d.channels = g.C; d.rows = g.M.data(); d.cols = g.N.data(); d.ksize = g.K;
    d.dtype = DECONV_F32; d.relax = 2.0f;
    size_t bound = 0;
    if (deconv_workspace_size(&d, &bound) != DECONV_OK) { printf("%s: unsupported\n", g.name); continue; }
    size_t mx = 0;
    std::vector<deconv_tune> all = tune_candidates(g.C);
    all.push_back(deconv_tune{0, 0, -1, 0, 0, 0, 0, 0, 0});
    for (deconv_tune t : all)
      for (int mb : {-1, 1, 24, 48, 80})
        for (int gen : {0, 1})
          for (int fr : {0, 1})
            for (int chn : {0, 1}) {
            t.l2_group_mb = mb; t.generic = gen; t.fused_rows = fr; t.chains = chn;
            Layout Lt;
            if (build_layout(&d, &Lt, &t) == DECONV_OK) {
              mx = std::max(mx, Lt.total);
              // The buffers the bulk copies and L2 prefetches read start on
              // kAlign boundaries and the workspace is padded to one, so a
              // prefetch widened to 16-byte granules stays inside its buffer.
              for (size_t o : {Lt.o_yt, Lt.o_d0, Lt.o_d1, Lt.o_Sa, Lt.o_Sb, Lt.o_xbuf, Lt.o_halo, Lt.total})
                if (o % kAlign != 0) {
                  printf("%s: offset %zu not on a %zu-byte boundary\n", g.name, o, kAlign);
                  ++misaligned;
                }
            }
          }
    printf("%s: bound %zu exact max %zu slack %zd %s\n", g.name, bound, mx, (ssize_t)(bound - mx), bound >= mx ? "ok" : "TOO SMALL");
    if (bound < mx) ++bad;
  }
  return bad + (misaligned ? 1 : 0);
}
