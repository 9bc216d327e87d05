// Patches of elements for the force sweep (host set-up of libsemgb).
//
// A patch is a small brick of neighbouring elements that one CTA evaluates together: it
// gathers the patch's distinct nodes once, sums the element forces that meet at each node
// in a fixed order inside the CTA, and writes each patch node once. Patches (not elements)
// are coloured so that no two patches of one colour share a node (Sec. IV-C's colouring,
// applied to groups of elements), which keeps the assembly free of atomics.
//
// Construction, for any conforming hexahedral mesh:
//   1. lattice coordinates by a walk across shared faces: an element reached across its
//      own +xi face of element e sits at coord(e) + (1, 0, 0), and so on for the six faces;
//      every connected component gets its own coordinates, shifted so that its lowest
//      cell is at 0 (first visit wins, so meshes whose element axes do not line up still
//      get a valid, if less compact, grouping);
//   2. bins of bx x by x bz lattice cells; a bin is a patch (bins holding more elements
//      than fit, possible only with inconsistent coordinates, are split in order);
//   3. greedy first-fit colouring of the patches in bin order over "shares a node";
//   4. per patch, its distinct nodes in order of first appearance (elements in lattice
//      order, points in natural order), the patch-local index of every local point and,
//      per patch node, the list of local points that meet there; patches with the same
//      local structure share one table (every interior brick of a structured mesh does);
//   5. an internal numbering of the nodes in which every patch finds its nodes in runs.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <string>
#include <unordered_map>
#include <vector>

#include "sem_internal.h"

namespace semgb {

namespace {

// Local point index of (i, j, k).
inline int lp(int n, int i, int j, int k) { return i + n * (j + n * k); }

// The four corner local points of face f (0: xi-, 1: xi+, 2: eta-, 3: eta+, 4: zeta-, 5: zeta+).
void face_corners(int n, int f, int out[4]) {
  const int N = n - 1;
  const int fixed = (f & 1) ? N : 0;
  int q = 0;
  for (int b = 0; b < 2; ++b)
    for (int a = 0; a < 2; ++a) {
      const int s = a * N, t = b * N;
      if (f < 2)
        out[q++] = lp(n, fixed, s, t);
      else if (f < 4)
        out[q++] = lp(n, s, fixed, t);
      else
        out[q++] = lp(n, s, t, fixed);
    }
}

struct FaceKey {
  int32_t v[4];
  bool operator==(const FaceKey& o) const { return std::memcmp(v, o.v, sizeof(v)) == 0; }
};

uint64_t hash_u16(const uint16_t* p, size_t n, uint64_t h) {
  for (size_t i = 0; i < n; ++i) {
    h ^= p[i];
    h *= 1099511628211ull;  // 64-bit FNV-1a prime
  }
  return h;
}

}  // namespace

int build_patches(int nspec, int n, int nglob, const int32_t* ibool, const PatchShape& shape, PatchPlan* plan,
                  std::string* err) {
  const int np = n * n * n;
  const int bx = std::max(1, shape.bx), by = std::max(1, shape.by), bz = std::max(1, shape.bz);
  const int cap = bx * by * bz;
  if (static_cast<long long>(cap) * np >= kPatchChain) {
    if (err) *err = "patch too large for 15-bit local indices";
    return -1;
  }

  // 1. faces keyed by their sorted corner nodes, grouped by the smallest corner node
  std::vector<FaceKey> key(static_cast<size_t>(nspec) * 6);
  int fc[6][4];
  for (int f = 0; f < 6; ++f) face_corners(n, f, fc[f]);
  std::vector<int> cnt(static_cast<size_t>(nglob) + 1, 0);
  for (int e = 0; e < nspec; ++e)
    for (int f = 0; f < 6; ++f) {
      FaceKey& k = key[static_cast<size_t>(e) * 6 + f];
      for (int q = 0; q < 4; ++q) k.v[q] = ibool[static_cast<size_t>(e) * np + fc[f][q]];
      std::sort(k.v, k.v + 4);
      cnt[k.v[0] + 1]++;
    }
  for (int g = 0; g < nglob; ++g) cnt[g + 1] += cnt[g];
  std::vector<int> face_at(static_cast<size_t>(cnt[nglob]));
  {
    std::vector<int> fill(cnt.begin(), cnt.end() - 1);
    for (int ef = 0; ef < nspec * 6; ++ef) face_at[fill[key[ef].v[0]]++] = ef;
  }
  // neighbour across face (e, f): the other element with the same face key, or -1
  auto neighbour = [&](int e, int f) -> int {
    const FaceKey& k = key[static_cast<size_t>(e) * 6 + f];
    for (int q = cnt[k.v[0]]; q < cnt[k.v[0] + 1]; ++q) {
      const int of = face_at[q];
      if (of / 6 != e && key[of] == k) return of / 6;
    }
    return -1;
  };

  // lattice coordinates by a breadth-first walk, one component after another
  std::vector<int> comp(nspec, -1);
  std::vector<int> cx(nspec, 0), cy(nspec, 0), cz(nspec, 0);
  std::vector<int> queue;
  queue.reserve(nspec);
  int ncomp = 0;
  static const int dir[6][3] = {{-1, 0, 0}, {1, 0, 0}, {0, -1, 0}, {0, 1, 0}, {0, 0, -1}, {0, 0, 1}};
  for (int s = 0; s < nspec; ++s) {
    if (comp[s] >= 0) continue;
    comp[s] = ncomp;
    queue.clear();
    queue.push_back(s);
    for (size_t h = 0; h < queue.size(); ++h) {
      const int e = queue[h];
      for (int f = 0; f < 6; ++f) {
        const int o = neighbour(e, f);
        if (o < 0 || comp[o] >= 0) continue;
        comp[o] = ncomp;
        cx[o] = cx[e] + dir[f][0];
        cy[o] = cy[e] + dir[f][1];
        cz[o] = cz[e] + dir[f][2];
        queue.push_back(o);
      }
    }
    // the component's lowest cell along each axis becomes 0, so that the bricks do not
    // depend on which element the walk started from
    int lo[3] = {cx[s], cy[s], cz[s]};
    for (int e : queue) {
      lo[0] = std::min(lo[0], cx[e]);
      lo[1] = std::min(lo[1], cy[e]);
      lo[2] = std::min(lo[2], cz[e]);
    }
    for (int e : queue) {
      cx[e] -= lo[0];
      cy[e] -= lo[1];
      cz[e] -= lo[2];
    }
    ++ncomp;
  }
  std::vector<FaceKey>().swap(key);
  std::vector<int>().swap(face_at);

  // 2. bins: sort elements by (component, bin z, bin y, bin x, z, y, x)
  auto fdiv = [](int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); };
  struct Item {
    int comp, bk, bj, bi, k, j, i, e;
  };
  std::vector<Item> items(nspec);
  for (int e = 0; e < nspec; ++e)
    items[e] = {comp[e], fdiv(cz[e], bz), fdiv(cy[e], by), fdiv(cx[e], bx), cz[e], cy[e], cx[e], e};
  std::sort(items.begin(), items.end(), [](const Item& a, const Item& b) {
    if (a.comp != b.comp) return a.comp < b.comp;
    if (a.bk != b.bk) return a.bk < b.bk;
    if (a.bj != b.bj) return a.bj < b.bj;
    if (a.bi != b.bi) return a.bi < b.bi;
    if (a.k != b.k) return a.k < b.k;
    if (a.j != b.j) return a.j < b.j;
    if (a.i != b.i) return a.i < b.i;
    return a.e < b.e;
  });
  std::vector<int> pel;                   // elements, patch after patch (bin order)
  std::vector<int> poff(1, 0);            // patch offsets into pel
  pel.reserve(nspec);
  for (int q = 0; q < nspec;) {
    int r = q + 1;
    while (r < nspec && items[r].comp == items[q].comp && items[r].bk == items[q].bk && items[r].bj == items[q].bj &&
           items[r].bi == items[q].bi)
      ++r;
    for (int s = q; s < r; s += cap) {
      for (int t = s; t < std::min(r, s + cap); ++t) pel.push_back(items[t].e);
      poff.push_back(static_cast<int>(pel.size()));
    }
    q = r;
  }
  const int npatch = static_cast<int>(poff.size()) - 1;

  // 3. greedy colouring of patches in bin order, over node -> patches incidence
  std::vector<int> pcount(static_cast<size_t>(nglob) + 1, 0);
  std::vector<int> stamp(nglob, -1);
  for (int P = 0; P < npatch; ++P)
    for (int q = poff[P]; q < poff[P + 1]; ++q)
      for (int p = 0; p < np; ++p) {
        const int g = ibool[static_cast<size_t>(pel[q]) * np + p];
        if (stamp[g] != P) {
          stamp[g] = P;
          pcount[g + 1]++;
        }
      }
  for (int g = 0; g < nglob; ++g) pcount[g + 1] += pcount[g];
  std::vector<int> patches_of(static_cast<size_t>(pcount[nglob]));
  {
    std::vector<int> fill(pcount.begin(), pcount.end() - 1);
    std::fill(stamp.begin(), stamp.end(), -1);
    for (int P = 0; P < npatch; ++P)
      for (int q = poff[P]; q < poff[P + 1]; ++q)
        for (int p = 0; p < np; ++p) {
          const int g = ibool[static_cast<size_t>(pel[q]) * np + p];
          if (stamp[g] != P) {
            stamp[g] = P;
            patches_of[fill[g]++] = P;
          }
        }
  }
  std::vector<int> pcolor(npatch, -1);
  std::vector<int> mark;
  int ncolors = 0;
  for (int P = 0; P < npatch; ++P) {
    for (int q = poff[P]; q < poff[P + 1]; ++q)
      for (int p = 0; p < np; ++p) {
        const int g = ibool[static_cast<size_t>(pel[q]) * np + p];
        for (int t = pcount[g]; t < pcount[g + 1]; ++t) {
          const int O = patches_of[t];
          if (O != P && pcolor[O] >= 0) {
            if (static_cast<int>(mark.size()) <= pcolor[O]) mark.resize(pcolor[O] + 1, -1);
            mark[pcolor[O]] = P;
          }
        }
      }
    int c = 0;
    while (c < static_cast<int>(mark.size()) && mark[c] == P) ++c;
    pcolor[P] = c;
    ncolors = std::max(ncolors, c + 1);
  }

  // sweep order: colour by colour, bin order inside a colour
  std::vector<int> porder(npatch);
  for (int P = 0; P < npatch; ++P) porder[P] = P;
  std::stable_sort(porder.begin(), porder.end(), [&](int a, int b) { return pcolor[a] < pcolor[b]; });

  PatchPlan& out = *plan;
  out = PatchPlan();
  out.ngll = n;
  out.npatch = npatch;
  out.ncolors = ncolors;
  out.color_off.assign(ncolors + 1, 0);
  for (int P = 0; P < npatch; ++P) out.color_off[pcolor[P] + 1]++;
  for (int c = 0; c < ncolors; ++c) out.color_off[c + 1] += out.color_off[c];
  out.elem.reserve(nspec);
  out.patch_off.assign(1, 0);
  out.node_off.assign(1, 0);
  out.table_of.reserve(npatch);

  // 4. node lists, first-touch flags, local-index and contribution tables
  std::vector<int> lidx(nglob, -1);  // patch-local index of a node while its patch is built
  std::vector<char> touched(nglob, 0);
  std::unordered_map<uint64_t, std::vector<int>> tables_by_hash;
  std::vector<uint16_t> lid;
  std::vector<int> nodes_tmp;
  for (int s = 0; s < npatch; ++s) {
    const int P = porder[s];
    const int m = poff[P + 1] - poff[P];
    nodes_tmp.clear();
    lid.assign(static_cast<size_t>(m) * np, 0);
    for (int le = 0; le < m; ++le) {
      const int e = pel[poff[P] + le];
      out.elem.push_back(e);
      for (int p = 0; p < np; ++p) {
        const int g = ibool[static_cast<size_t>(e) * np + p];
        if (lidx[g] < 0) {
          lidx[g] = static_cast<int>(nodes_tmp.size());
          nodes_tmp.push_back(g);
        }
        lid[static_cast<size_t>(le) * np + p] = static_cast<uint16_t>(lidx[g]);
      }
    }
    const int nn = static_cast<int>(nodes_tmp.size());
    // contributions per patch node, ascending local point index c = le*np + p. A node met
    // by one local point only ("exclusive": inside one element of the patch) is flagged in
    // a bit mask over the local points; the others ("shared") get kPatchSlots fixed slots
    // each, in first-appearance order (unused slots kPatchNoSlot; a node met by more local
    // points continues in another group of slots, named by the last slot of the group as
    // kPatchChain | index of the next group)
    std::vector<uint16_t> first_q(nn), slots;
    std::vector<uint32_t> excl((lid.size() + 31) / 32, 0u);
    int nshared = 0;
    {
      std::vector<std::vector<uint16_t>> con(nn);
      for (size_t c = 0; c < lid.size(); ++c) con[lid[c]].push_back(static_cast<uint16_t>(c));
      for (int t = 0; t < nn; ++t) {
        first_q[t] = con[t][0];
        if (con[t].size() == 1) excl[con[t][0] / 32] |= 1u << (con[t][0] % 32);
        else ++nshared;
      }
      slots.assign(static_cast<size_t>(nshared) * kPatchSlots, kPatchNoSlot);
      int sidx = 0;
      for (int t = 0; t < nn; ++t) {
        if (con[t].size() == 1) continue;
        size_t g = static_cast<size_t>(sidx++);  // slot group being filled
        size_t k = 0;
        for (size_t q = 0; q < con[t].size(); ++q) {
          const bool last_slot = k == kPatchSlots - 1, more = q + 1 < con[t].size();
          if (last_slot && more) {  // chain to a new group at the end of the table
            const size_t ng = slots.size() / kPatchSlots;
            slots[g * kPatchSlots + k] = static_cast<uint16_t>(kPatchChain | ng);
            slots.resize(slots.size() + kPatchSlots, kPatchNoSlot);
            g = ng;
            k = 0;
          }
          slots[g * kPatchSlots + k++] = con[t][q];
        }
      }
      if (slots.size() / kPatchSlots > kPatchChain) {
        if (err) *err = "patch contribution table too large";
        return -1;
      }
    }
    for (int t = 0; t < nn; ++t) {
      const int g = nodes_tmp[t];
      uint32_t w = static_cast<uint32_t>(g);
      if (!touched[g]) {
        touched[g] = 1;
        w |= kFirstTouchBit;
      }
      out.nodes.push_back(w);
      lidx[g] = -1;
    }
    out.max_nodes = std::max(out.max_nodes, nn);
    out.max_elems = std::max(out.max_elems, m);
    out.patch_off.push_back(static_cast<int>(out.elem.size()));
    out.node_off.push_back(static_cast<int>(out.nodes.size()));
    // shared table: same element count, node count and local indices
    const uint64_t h = hash_u16(lid.data(), lid.size(), 1469598103934665603ull ^ (static_cast<uint64_t>(m) << 32) ^ nn);
    int tid = -1;
    auto& cands = tables_by_hash[h];
    for (int t : cands) {
      if (out.tab_nelem[t] == m && out.tab_nnode[t] == nn &&
          std::equal(lid.begin(), lid.end(), out.lid.begin() + out.tab_lid_off[t])) {
        tid = t;
        break;
      }
    }
    if (tid < 0) {
      tid = static_cast<int>(out.tab_nelem.size());
      cands.push_back(tid);
      out.tab_nelem.push_back(m);
      out.tab_nnode.push_back(nn);
      out.tab_nshared.push_back(nshared);
      out.tab_lid_off.push_back(static_cast<int>(out.lid.size()));
      out.lid.insert(out.lid.end(), lid.begin(), lid.end());
      out.tab_csr_off.push_back(static_cast<int>(out.csr.size()));
      out.csr.insert(out.csr.end(), slots.begin(), slots.end());
      out.tab_excl_off.push_back(static_cast<int>(out.excl.size()));
      out.excl.insert(out.excl.end(), excl.begin(), excl.end());
      out.tab_first_off.push_back(static_cast<int>(out.first_q.size()));
      out.first_q.insert(out.first_q.end(), first_q.begin(), first_q.end());
    }
    out.table_of.push_back(tid);
  }

  // 5. internal node numbering: the nodes a patch touches first (in sweep order) get the
  //    next consecutive ids, grouped by the set of patches that share them (the patch's own
  //    interior, then each shared face, edge and corner group together, so that the
  //    neighbours that read them find them in runs), in first appearance order inside a
  //    group
  {
    std::vector<int> sweep_pos(npatch);
    for (int s2 = 0; s2 < npatch; ++s2) sweep_pos[porder[s2]] = s2;
    out.node_new.assign(nglob, -1);
    int next = 0;
    std::vector<std::pair<std::vector<int>, int>> keyed;  // (sharers in sweep order, appearance)
    for (int s2 = 0; s2 < npatch; ++s2) {
      keyed.clear();
      for (int t = out.node_off[s2]; t < out.node_off[s2 + 1]; ++t) {
        if (!(out.nodes[t] & kFirstTouchBit)) continue;
        const int g = static_cast<int>(out.nodes[t] & ~kFirstTouchBit);
        std::vector<int> sh;
        for (int q = pcount[g]; q < pcount[g + 1]; ++q) sh.push_back(sweep_pos[patches_of[q]]);
        std::sort(sh.begin(), sh.end());
        keyed.emplace_back(std::move(sh), t);
      }
      std::stable_sort(keyed.begin(), keyed.end(), [](const auto& a, const auto& b) {
        if (a.first.size() != b.first.size()) return a.first.size() < b.first.size();
        return a.first < b.first;
      });
      for (const auto& kv : keyed) out.node_new[out.nodes[kv.second] & ~kFirstTouchBit] = next++;
    }
    if (next != nglob) {
      if (err) *err = "internal numbering does not cover every node";
      return -1;
    }
  }

  // exhaustive check: inside one colour no node is touched by two patches
  std::vector<int> seen_color(nglob, -1), seen_patch(nglob, -1);
  for (int c = 0; c < ncolors; ++c)
    for (int s = out.color_off[c]; s < out.color_off[c + 1]; ++s)
      for (int t = out.node_off[s]; t < out.node_off[s + 1]; ++t) {
        const int g = static_cast<int>(out.nodes[t] & ~kFirstTouchBit);
        if (seen_color[g] == c && seen_patch[g] != s) {
          if (err) *err = "patch colouring failed at node " + std::to_string(g);
          return -1;
        }
        seen_color[g] = c;
        seen_patch[g] = s;
      }
  return 0;
}

}  // namespace semgb
