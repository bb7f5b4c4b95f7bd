"""The neighbour list's chunk count (csrc/sph_internal.cuh, list_chunks) fits
every split of a full list: the fluid part fills chunks from the front, the
boundary part from the back, two entries per chunk, and for every list size
the library accepts (8..1024) and every nf + nb <= max_neibs the two parts
never share a chunk.  The formula is read from the header, not restated."""
import os
import re

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                      "paper_2207_11328_gb300", "csrc", "sph_internal.cuh")


def _list_chunks():
    src = open(HEADER).read()
    m = re.search(r"constexpr uint32_t list_chunks\(uint32_t max_neibs\) \{ return ([^;]+); \}", src)
    assert m, "list_chunks not found"
    expr = m.group(1).replace("u", "").replace("/", "//")
    return lambda max_neibs: eval(expr, {}, {"max_neibs": max_neibs})


def test_every_split_fits_without_sharing_a_chunk():
    chunks = _list_chunks()
    for m in range(8, 1025):
        c = chunks(m)
        for nf in range(m + 1):
            nb = m - nf  # the fullest lists; shorter ones use fewer chunks
            used_f = (nf + 1) // 2          # chunks 0 .. used_f - 1
            used_b = (nb + 1) // 2          # chunks c - used_b .. c - 1
            assert used_f + used_b <= c, (m, nf, nb, c)


def test_chunk_count_is_tight():
    # one chunk fewer would not fit two odd parts of a full even-sized list
    chunks = _list_chunks()
    for m in range(8, 1025, 2):
        assert (1 + 1) // 2 + (m - 1 + 1) // 2 == chunks(m)


def test_exact_list_parts_fit():
    # skin list: the step's exact list in chunks of four, fluid part from chunk 0, boundary
    # part from chunk exact_bnd_chunk(max_neibs), 2 * exact_bnd_chunk chunks per particle
    src = open(HEADER).read()
    m = re.search(r"constexpr uint32_t exact_bnd_chunk\(uint32_t max_neibs\) \{ return ([^;]+); \}", src)
    assert m, "exact_bnd_chunk not found"
    expr = m.group(1).replace("u", "").replace("/", "//")
    kxb = lambda max_neibs: eval(expr, {}, {"max_neibs": max_neibs})  # noqa: E731
    for mn in range(8, 1025):
        k = kxb(mn)
        assert (mn + 3) // 4 <= k          # a fluid part of up to max_neibs entries
        assert k + (mn + 3) // 4 <= 2 * k  # a boundary part of up to max_neibs entries
