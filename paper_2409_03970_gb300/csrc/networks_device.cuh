// Comparator networks for the column sort (Sec. 2.3, Table 1), generated at
// compile time.
//
// A network is a list of comparators (lo, hi), lo < hi: afterwards
// v[lo] <= v[hi].  Three families, for widths 4, 8, 16 and 32:
//   NET_BITONIC  Batcher's bitonic sorter in the flip form (each merge of two
//                runs of m compares wire i with its mirror 2m-1-i, then
//                half-cleans at distances m/2 .. 1): 6 / 24 / 80 / 240.
//   NET_ODDEVEN  Batcher's odd-even merge sort, phase p merging runs of p
//                into runs of 2p: 5 / 19 / 63 / 191.
//   NET_BEST     the fewest comparators known (Table 1, last column):
//                widths 4 and 8 take the odd-even networks (5 and 19 are
//                optimal); 16 takes M. W. Green's 60-comparator network;
//                32 sorts both halves with Green's network and merges them
//                with the last odd-even phase (2 * 60 + 65 = 185).
// The same constexpr lists drive the device column sorts (fully unrolled,
// every index a constant, so the keys stay in registers) and are exported to
// the host for checking.
#pragma once

namespace nsort {

enum NetFamily { NET_BITONIC = 0, NET_ODDEVEN = 1, NET_BEST = 2 };

constexpr int NET_MAX_COMPARATORS = 256;

struct CmpList {
  int n = 0;
  unsigned char lo[NET_MAX_COMPARATORS] = {};
  unsigned char hi[NET_MAX_COMPARATORS] = {};
  __host__ __device__ constexpr void add(int a, int b) {
    lo[n] = (unsigned char)a;
    hi[n] = (unsigned char)b;
    ++n;
  }
};

// Green's network on wires [base, base + 16): four layers compare the wires
// whose indices differ in one bit (a 4-cube), six more layers finish.
__host__ __device__ constexpr void add_green16(CmpList &l, int base) {
  for (int bit = 1; bit < 16; bit <<= 1)
    for (int i = 0; i < 16; ++i)
      if (!(i & bit)) l.add(base + i, base + (i | bit));
  constexpr int tail[28][2] = {
      {5, 10}, {6, 9}, {3, 12}, {13, 14}, {7, 11}, {1, 2}, {4, 8},      // layer 5
      {1, 4}, {7, 13}, {2, 8}, {11, 14}, {5, 6}, {9, 10},               // layer 6
      {2, 4}, {11, 13}, {3, 8}, {7, 12},                                // layer 7
      {6, 8}, {10, 12}, {3, 5}, {7, 9},                                 // layer 8
      {3, 4}, {5, 6}, {7, 8}, {9, 10}, {11, 12},                        // layer 9
      {6, 7}, {8, 9}};                                                  // layer 10
  for (int c = 0; c < 28; ++c) l.add(base + tail[c][0], base + tail[c][1]);
}

// Odd-even merge phase p on w wires: merges every pair of adjacent sorted
// runs of p into a sorted run of 2p.  Stage k = p compares each wire x with
// x mod 2p < p against x + p; each later stage k = p/2, .., 1 compares each
// wire x with x mod 2k >= k against x + k.  Comparators whose two wires fall
// in different runs of 2p are left out.
__host__ __device__ constexpr void add_oddeven_phase(CmpList &l, int w, int p) {
  for (int k = p; k >= 1; k >>= 1)
    for (int j = k % p; j + k < w; j += 2 * k)
      for (int i = 0; i < k && i + j + k < w; ++i)
        if ((i + j) / (2 * p) == (i + j + k) / (2 * p)) l.add(i + j, i + j + k);
}

__host__ __device__ constexpr CmpList make_network(int family, int w) {
  CmpList l{};
  if (w != 4 && w != 8 && w != 16 && w != 32) return l;
  if (family == NET_BITONIC) {
    for (int m = 1; m < w; m <<= 1) {
      for (int i = 0; i < w; ++i)
        if (!(i & m)) l.add(i, i ^ (2 * m - 1));        // flip: i against its mirror
      for (int d = m >> 1; d >= 1; d >>= 1)
        for (int i = 0; i < w; ++i)
          if (!(i & d)) l.add(i, i | d);                // half-cleaners
    }
  } else if (family == NET_ODDEVEN || (family == NET_BEST && w <= 8)) {
    for (int p = 1; p < w; p <<= 1) add_oddeven_phase(l, w, p);
  } else if (family == NET_BEST) {
    add_green16(l, 0);
    if (w == 32) {
      add_green16(l, 16);
      add_oddeven_phase(l, 32, 16);
    }
  }
  return l;
}

}  // namespace nsort
