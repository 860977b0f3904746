"""The oracle's pins must catch plausible mistakes.

Each case plants one mistake in a private copy of the oracle's C source (a
dropped alignment, an off-by-one index, a wrong operand), builds it, and
runs the pin tests against it in a subprocess: they must fail.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "mrn_oracle.c")

MUTANTS = {
    "aosoa_no_align": ("start = align_up(end, s->store_align[k]);", "start = end;"),
    "begin_align_4": ("s->begin_off = align_up(cur, 8);", "s->begin_off = align_up(cur, 4);"),
    "group_not_aligned": ("uint64_t goff = align_up(cur, galign);", "uint64_t goff = cur;"),
    "no_tail_padding": ("*size_out = align_up(cur, al);", "*size_out = cur;"),
    "offsets_off_by_one": ("wr(off + (i + 1) * s->off_size, run, s->off_size);",
                           "wr(off + i * s->off_size, run, s->off_size);"),
    "wrong_record": ("memcpy(col_addr(s, dst, c, i), col_addr(s, src, c, i), s->col_size[c]);",
                     "memcpy(col_addr(s, dst, c, i), col_addr(s, src, c, (i + 1) % n), s->col_size[c]);"),
    "soa_align_64": ("start = align_up(end, 128);", "start = align_up(end, 64);"),
    "child_wrong_column": ("src->pool + (beg + k) * ch->stride + ch->col_aos_off[cc]",
                           "src->pool + (beg + k) * ch->stride + ch->col_aos_off[0]"),
    "aosoa_slot_swapped": ("(i % v->block) * es;", "((v->block - 1 - i % v->block)) * es;"),
    "jagged_aosoa_regions_as_soa": ("static int parent_regions(const orc_schema* s, int kind) { return kind == ORC_AOSOA ? 1 : s->nstore; }",
                                    "static int parent_regions(const orc_schema* s, int kind) { return s->nstore; }"),
    "f2f_children_dropped": ("memcpy(child_col_ptr(s, dst, cc), child_col_ptr(s, src, cc), src->m * ch->col_es[cc]);",
                             "(void)cc;"),
    "interleaved_stride_as_size": ("s->col_es[s->ncols] = s->store_es[s->nstore - 1];",
                                   "s->col_es[s->ncols] = size;"),
    "interleaved_element_offset_dropped": ("s->col_sub[s->ncols] = inter ? (uint32_t)k * size : 0;",
                                           "s->col_sub[s->ncols] = 0;"),
    "nested_offsets_not_summed": ("          run1 += len1;\n", "\n"),
    "nested_grandchild_from_run_start": ("src->gpool + (beg1 + q) * gc->stride + gc->col_aos_off[g]",
                                         "src->gpool + q * gc->stride + gc->col_aos_off[g]"),
    "nested_grandchild_regions_dropped": ("return fm_region_bytes(s->child, ORC_SOA, 0, m, m2, 0, q - P - 1);",
                                          "return fm_region_bytes(s->child, ORC_SOA, 0, m, 0, 0, q - P - 1);"),
    "nested_begin_from_next_offset": ("        wr(c + ch->begin_off, a, 8);", "        wr(c + ch->begin_off, b, 8);"),
    "jagged_offsets_item_as_storage_index": ("static int offsets_item(const orc_schema* s, int kind) { return kind == ORC_AOSOA ? 1 : s->ncols; }",
                                             "static int offsets_item(const orc_schema* s, int kind) { return kind == ORC_AOSOA ? 1 : s->nstore; }"),
    "interleaved_block_row_as_element": ("end = start + (uint64_t)B * s->store_es[k];",
                                         "end = start + (uint64_t)B * s->store_align[k];"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, name
    mut = tmp_path / "mutant.c"
    mut.write_text(src.replace(old, new))
    lib = tmp_path / "libmutant.so"
    subprocess.run(["gcc", "-O1", "-shared", "-fPIC", str(mut), "-o", str(lib)], check=True)
    env = dict(os.environ, MRN_ORACLE_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, "pins did not catch mutant %s" % name
    assert "failed" in r.stdout
