"""The library's host symbolic analysis (``csrc/symbolic.cpp``), run on the CPU through a test-only
shim (``tests/host_symbolic_shim.cpp``), without a GPU.

- Local structure against the oracle, exactly: counts of fine cells, near lumps and far lumps, the
  cell -> local row map, and the block pattern of A_i (Section 4).
- The assembly lists evaluated on the host equal the oracle's A_i = R_i A R_i^T (Eq. 4.1, Appendix B)
  within 1e-12 per block row.  Every slot is a far-box block sum C(J, J') and/or signed blocks of A.
- The wavefront levels are a valid schedule for both sweeps (Section 2: the forward sweep needs
  every lower neighbour first, the backward sweep every upper one), each row at its earliest level.
- The factor stream is a valid schedule too.  Chunks decoded from their bytes cover every row once
  per sweep, in the level order, with the row's own column list.  No row reads a row of a level that
  has not closed.  Every chunk fits the subdomain's chunk capacity.
- The pack map sends every factor slot of A_i's pattern to exactly one place in the stream.
"""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle as O
from paper_1401_7227_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1401_7227_gb300", "csrc")
CHUNK_MIN, CHUNK_MAX = 8192, 24576     # kStreamChunkMin / kStreamChunkMax of the library
FINE_BLOCK_BYTES = {0: 72, 1: 36, 2: 20}  # FP64, FP32, FP16 + exponent fine-row blocks

GEOMS = {
    "cfg1": (O.Geometry(10, 10, 5, 2, 2, 1, ov=1), 1),
    "ragged": (O.Geometry(9, 7, 6, 3, 2, 2, ov=1, near_width=1, cnear=(2, 3, 2)), 2),
    "cfar": (O.Geometry(12, 6, 5, 3, 1, 1, ov=2, near_width=2, cnear=(3, 2, 2), far_mode=2, cfar=(4, 3, 5)), 3),
    "nofar": (O.Geometry(8, 8, 4, 2, 2, 1, ov=1, near_width=2, far_mode=0), 4),
    "nonear": (O.Geometry(8, 8, 4, 2, 2, 1, ov=0, near_width=0, far_mode=1), 5),
    "k1": (O.Geometry(6, 5, 4, 1, 1, 1, ov=0, near_width=0), 6),
    "k32": (O.Geometry(16, 16, 8, 4, 4, 2, ov=1), 7),
    "tall": (O.Geometry(5, 4, 40, 1, 2, 3, ov=2, near_width=2, cnear=(2, 2, 4)), 8),
    "wide_near": (O.Geometry(14, 11, 3, 2, 3, 1, ov=0, near_width=3, cnear=(3, 2, 3)), 9),
    "far_small": (O.Geometry(12, 12, 6, 3, 3, 1, ov=1, near_width=1, far_mode=2, cfar=(2, 2, 3)), 10),
    "ov_wide": (O.Geometry(10, 9, 8, 2, 3, 2, ov=3, near_width=2, cnear=(4, 4, 4)), 11),
    "line": (O.Geometry(1, 1, 30, 1, 1, 4, ov=1, near_width=2, cnear=(1, 1, 2)), 12),
    # edge cases: one-cell-wide boxes, an overlap or a near ring that covers the grid, near boxes
    # larger than the grid, one-cell and whole-grid far boxes, no near and no far field
    "thin_x": (O.Geometry(6, 4, 3, 6, 1, 1, ov=1, near_width=2), 16),
    "thin_all": (O.Geometry(3, 3, 3, 3, 3, 3, ov=0, near_width=1, cnear=(1, 1, 1)), 17),
    "ov_covers": (O.Geometry(6, 5, 4, 2, 1, 1, ov=10, near_width=2), 18),
    "ring_covers": (O.Geometry(6, 5, 4, 2, 2, 1, ov=0, near_width=20), 19),
    "cnear_big": (O.Geometry(6, 5, 4, 2, 1, 1, ov=0, near_width=2, cnear=(50, 50, 50)), 20),
    "cfar_one": (O.Geometry(6, 5, 4, 2, 1, 1, ov=0, near_width=1, far_mode=2, cfar=(1, 1, 1)), 21),
    "cfar_big": (O.Geometry(6, 5, 4, 2, 2, 1, ov=0, near_width=1, far_mode=2, cfar=(40, 40, 40)), 22),
    "cnear_odd": (O.Geometry(7, 9, 5, 2, 3, 1, ov=1, near_width=3, cnear=(3, 4, 5), far_mode=2, cfar=(5, 2, 3)), 23),
    "z_split": (O.Geometry(4, 4, 12, 1, 1, 6, ov=1, near_width=2), 24),
    "nothing": (O.Geometry(6, 6, 3, 3, 3, 1, ov=0, near_width=0, far_mode=0), 25),
}
# levels of several hundred fine rows: more than the largest chunk capacity, so levels are split
WIDE = (O.Geometry(40, 40, 8, 1, 1, 1, ov=0, near_width=0, far_mode=0), 15)


@pytest.fixture(scope="module")
def hs(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no g++")
    out = str(tmp_path_factory.mktemp("hs") / "libhs.so")
    cuda_inc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")
    subprocess.run([cxx, "-std=c++17", "-O1", "-fPIC", "-shared", f"-I{os.path.join(ROOT, 'include')}", f"-I{CSRC}",
                    f"-I{cuda_inc}", os.path.join(CSRC, "symbolic.cpp"),
                    os.path.join(ROOT, "tests", "host_symbolic_shim.cpp"), "-o", out, "-lpthread"], check=True)
    lib = C.CDLL(out)
    lib.hs_create.restype = C.c_void_p
    lib.hs_create.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_char_p,
                              C.c_int, C.c_int]
    lib.hs_destroy.argtypes = [C.c_void_p]
    lib.hs_get.restype = C.c_longlong
    lib.hs_get.argtypes = [C.c_void_p, C.c_int, C.c_char_p, C.c_void_p]
    lib.hs_check_pattern.argtypes = [C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_char_p, C.c_int]
    return lib


class Sym:
    """The symbolic structure of one system, read through the shim."""

    DTYPES = {"chunk_off": np.int64, "pk_off_f": np.int64, "pk_off_c": np.int64, "stream": np.uint8}

    def __init__(self, lib, g, s, prec=0, colsum=1, lump32=0, chunk_force=0):
        geo = np.array([g.nx, g.ny, g.nz, g.px, g.py, g.pz, g.ov, g.near_width, *g.cnear, g.far_mode,
                        *(g.cfar if g.far_mode == 2 else (1, 1, 1))], dtype=np.int32)
        rp = np.ascontiguousarray(s.row_ptr, dtype=np.int32)
        ci = np.ascontiguousarray(s.col_idx, dtype=np.int32)
        err = C.create_string_buffer(256)
        self.lib = lib
        self.h = lib.hs_create(geo.ctypes.data, s.n_cells, s.nnzb, rp.ctypes.data, ci.ctypes.data, prec, lump32, colsum,
                               err, 256, chunk_force)
        assert self.h, err.value.decode()

    def __del__(self):
        if getattr(self, "h", None):
            self.lib.hs_destroy(self.h)

    def get(self, s, what):
        n = self.lib.hs_get(self.h, s, what.encode(), None)
        assert n >= 0, what
        a = np.empty(n, dtype=self.DTYPES.get(what, np.int32))
        self.lib.hs_get(self.h, s, what.encode(), a.ctypes.data)
        return a

    def info(self, s):
        return dict(zip(("n", "nf", "nn", "nfar", "nslot", "nlev", "chunk_cap", "n_fwd_chunks"), self.get(s, "info")))


def assembled_values(sym, s, vals):
    """Slot values of A_s from the assembly lists: C(J, J') where a slot has one, plus its signed
    blocks of A (~e: subtracted)."""
    cptr, cloc = sym.get(-1, "cptr"), sym.get(-1, "cloc")
    cval = np.zeros((max(len(cptr) - 1, 0), 3, 3))
    if len(cloc):
        np.add.at(cval, np.repeat(np.arange(len(cptr) - 1), np.diff(cptr)), vals[cloc])
    aptr, aloc, acs = sym.get(s, "aptr"), sym.get(s, "aloc"), sym.get(s, "acs")
    out = np.zeros((len(acs), 3, 3))
    has_c = acs >= 0
    out[has_c] = cval[acs[has_c]]
    sign = np.where(aloc >= 0, 1.0, -1.0)
    idx = np.where(aloc >= 0, aloc, ~aloc)
    np.add.at(out, np.repeat(np.arange(len(acs)), np.diff(aptr)), sign[:, None, None] * vals[idx])
    return out


def rowwise_rel(a, b, rp):
    worst = 0.0
    for p in range(len(rp) - 1):
        d = np.linalg.norm(a[rp[p]:rp[p + 1]] - b[rp[p]:rp[p + 1]])
        worst = max(worst, d / max(np.linalg.norm(b[rp[p]:rp[p + 1]]), 1e-300))
    return worst


@pytest.mark.parametrize("name", list(GEOMS))
def test_local_structure_and_assembly_match_oracle(hs, name):
    g, seed = GEOMS[name]
    s = synth.grid_jacobian(g.nx, g.ny, g.nz, seed)
    sym = Sym(hs, g, s)
    pc = O.Precond(g, s.row_ptr, s.col_idx, s.vals)
    assert sym.get(-1, "n_sub")[0] == g.n_sub
    for sd in range(g.n_sub):
        inf = sym.info(sd)
        assert (inf["nf"], inf["nn"], inf["nfar"]) == pc.sub_counts(sd)
        assert inf["n"] == pc.sub_n(sd)
        np.testing.assert_array_equal(sym.get(sd, "map"), pc.sub_map(sd))
        orp, oci, ov = pc.sub_matrix(sd)
        np.testing.assert_array_equal(sym.get(sd, "prp"), orp)
        np.testing.assert_array_equal(sym.get(sd, "pci"), oci)
        assert rowwise_rel(assembled_values(sym, sd, s.vals), ov, orp) <= 1e-12


def levels_of(sym, sd):
    rop, lv0 = sym.get(sd, "row_of_pos"), sym.get(sd, "lv_pos0")
    level = np.empty(len(rop), dtype=np.int64)
    for l in range(len(lv0) - 1):
        level[rop[lv0[l]:lv0[l + 1]]] = l
    return level


@pytest.mark.parametrize("name", list(GEOMS))
def test_wavefront_levels_are_an_earliest_valid_schedule(hs, name):
    g, seed = GEOMS[name]
    s = synth.grid_jacobian(g.nx, g.ny, g.nz, seed)
    sym = Sym(hs, g, s)
    for sd in range(g.n_sub):
        inf = sym.info(sd)
        n, nf = inf["n"], inf["nf"]
        rp, ci, pdiag = sym.get(sd, "prp"), sym.get(sd, "pci"), sym.get(sd, "pdiag")
        rop, lv0 = sym.get(sd, "row_of_pos"), sym.get(sd, "lv_pos0")
        assert len(lv0) == inf["nlev"] + 1 and lv0[0] == 0 and lv0[-1] == n
        np.testing.assert_array_equal(np.sort(rop), np.arange(n))
        level = levels_of(sym, sd)
        for p in range(n):
            assert ci[pdiag[p]] == p
            lower, upper = ci[rp[p]:pdiag[p]], ci[pdiag[p] + 1:rp[p + 1]]
            assert np.all(level[lower] < level[p]), (sd, p)            # forward sweep
            assert np.all(level[upper] > level[p]), (sd, p)            # backward sweep
            assert level[p] == (level[lower].max() + 1 if len(lower) else 0), (sd, p)  # earliest level
        for l in range(inf["nlev"]):   # within a level the fine rows come first
            is_fine = rop[lv0[l]:lv0[l + 1]] < nf
            assert not np.any(is_fine[np.argmax(~is_fine):]) or np.all(is_fine)
        # fine and lump indices number the rows in position order
        fid, cid = sym.get(sd, "fidx_of_row"), sym.get(sd, "cidx_of_row")
        np.testing.assert_array_equal(fid[rop[rop < nf]], np.arange(nf))
        np.testing.assert_array_equal(cid[rop[rop >= nf]], np.arange(n - nf))
        assert np.all(fid[nf:] == -1) and np.all(cid[:nf] == -1)


def al16(x):
    return (x + 15) // 16 * 16


def decode_chunks(sym, sd, prec, lump32=0):
    """Chunks of subdomain sd's factor stream: (fwd, f0, nf, c0, nc, last, fine rows' columns, lump
    rows' columns, value offsets of the fine and lump blocks, bytes)."""
    stream, off, nbytes = sym.get(sd, "stream"), sym.get(sd, "chunk_off"), sym.get(sd, "chunk_bytes")
    nfwd = sym.info(sd)["n_fwd_chunks"]
    fbb = FINE_BLOCK_BYTES[prec]
    out = []
    for i, (o, nb) in enumerate(zip(off, nbytes)):
        fwd = i < nfwd
        hdr = stream[o:o + 32].view(np.int32)
        f0, nf, c0, nc, nef, nec, flags, b = (int(x) for x in hdr)
        assert b == nb
        w = o + 32
        groups = []
        for cnt, ne, bb in ((nf, nef, fbb), (nc, nec, 36 if lump32 and prec else 72)):
            ptr = stream[w:w + 4 * (cnt + 1)].view(np.int32)
            assert ptr[0] == 0 and ptr[-1] == ne
            w += al16(4 * (cnt + 1))
            col = stream[w:w + 4 * ne].view(np.int32)
            w += al16(4 * ne)
            vals = [w + bb * e for e in range(ne)]
            w += al16(bb * ne)
            if not fwd:
                vals += [w + bb * k for k in range(cnt)]
                w += al16(bb * cnt)
            groups.append(([col[ptr[k]:ptr[k + 1]] for k in range(cnt)], vals))
        assert w == o + nb, "chunk size does not match its layout"
        out.append(dict(fwd=fwd, f0=f0, nf=nf, c0=c0, nc=nc, last=bool(flags & 1), fcols=groups[0][0],
                        ccols=groups[1][0], fvals=groups[0][1], cvals=groups[1][1], bytes=nb))
    return out


@pytest.mark.parametrize("prec,lump32", [(0, 0), (1, 0), (2, 0), (1, 1), (2, 1)])
@pytest.mark.parametrize("name", ["cfg1", "ragged", "cfar", "k32", "tall", "far_small", "ov_wide", "wide"])
def test_factor_stream_is_a_valid_schedule(hs, name, prec, lump32):
    g, seed = WIDE if name == "wide" else GEOMS[name]
    s = synth.grid_jacobian(g.nx, g.ny, g.nz, seed)
    check_stream(Sym(hs, g, s, prec=prec, lump32=lump32), g, prec, lump32)


@pytest.mark.parametrize("prec,lump32", [(0, 0), (1, 1)])
@pytest.mark.parametrize("chunk_kb", [8, 12, 24])
@pytest.mark.parametrize("name", ["cfg1", "k32", "wide"])
def test_forced_chunk_capacity_gives_a_valid_schedule(hs, name, chunk_kb, prec, lump32):
    """The tiling tuner's capacities (ASM_TUNE_CHUNK_KB): every subdomain gets exactly the capacity
    asked for (no row of these geometries needs more), chunks stay within it, and the stream is
    still a valid schedule with the same rows as under the rule."""
    g, seed = WIDE if name == "wide" else GEOMS[name]
    s = synth.grid_jacobian(g.nx, g.ny, g.nz, seed)
    sym = Sym(hs, g, s, prec=prec, lump32=lump32, chunk_force=chunk_kb * 1024)
    rule = Sym(hs, g, s, prec=prec, lump32=lump32)
    for sd in range(g.n_sub):
        assert sym.info(sd)["chunk_cap"] == chunk_kb * 1024
        np.testing.assert_array_equal(sym.get(sd, "row_of_pos"), rule.get(sd, "row_of_pos"))
    check_stream(sym, g, prec, lump32)


def test_forced_chunk_capacity_out_of_range_is_refused(hs):
    g, seed = GEOMS["cfg1"]
    s = synth.grid_jacobian(g.nx, g.ny, g.nz, seed)
    for bad in (4096, 10000, 28672):
        with pytest.raises(AssertionError, match="capacity out of range"):
            Sym(hs, g, s, chunk_force=bad)


def check_stream(sym, g, prec, lump32):
    for sd in range(g.n_sub):
        inf = sym.info(sd)
        n, nf, cap = inf["n"], inf["nf"], inf["chunk_cap"]
        assert CHUNK_MIN <= cap <= CHUNK_MAX and cap % 4096 == 0
        rp, ci, pdiag = sym.get(sd, "prp"), sym.get(sd, "pci"), sym.get(sd, "pdiag")
        rop, fid, cid = sym.get(sd, "row_of_pos"), sym.get(sd, "fidx_of_row"), sym.get(sd, "cidx_of_row")
        row_of_f, row_of_c = rop[rop < nf], rop[rop >= nf]
        off, nbytes = sym.get(sd, "chunk_off"), sym.get(sd, "chunk_bytes")
        assert off[0] == 0 and np.all(off % 16 == 0) and np.all(nbytes <= cap)
        np.testing.assert_array_equal(off[1:], off[:-1] + nbytes[:-1])
        assert off[-1] + nbytes[-1] == len(sym.get(sd, "stream"))
        chunks = decode_chunks(sym, sd, prec, lump32)
        level = levels_of(sym, sd)
        for fwd in (True, False):
            seen = np.zeros(n, dtype=np.int64)
            closed = np.zeros(n, dtype=bool)   # rows of the levels whose last chunk has passed
            pending = []
            last_level = None
            for ch in (c for c in chunks if c["fwd"] == fwd):
                rows = [int(row_of_f[ch["f0"] + k]) for k in range(ch["nf"])] + \
                       [int(row_of_c[ch["c0"] + k]) for k in range(ch["nc"])]
                lv = {int(level[p]) for p in rows}
                assert len(lv) == 1, "a chunk mixes levels"
                lv = lv.pop()
                if last_level is not None:
                    assert lv == last_level or (lv > last_level if fwd else lv < last_level)
                last_level = lv
                for p, cols in zip(rows, list(ch["fcols"]) + list(ch["ccols"])):
                    seen[p] += 1
                    want = ci[rp[p]:pdiag[p]] if fwd else ci[pdiag[p] + 1:rp[p + 1]]
                    got = np.array([row_of_f[c] if c >= 0 else row_of_c[~c] for c in cols], dtype=np.int64)
                    np.testing.assert_array_equal(got, want)
                    assert np.all(closed[got]), "a row reads a row of an unfinished level"
                pending += rows
                if ch["last"]:
                    closed[pending] = True
                    pending = []
            assert not pending
            np.testing.assert_array_equal(seen, np.ones(n))
        # pack map: every slot of a fine row once (L, U, and D^-1 from the diagonal slot), likewise
        # for the lump rows, each to its own value block of the stream
        for grp, rows in (("f", np.arange(nf)), ("c", np.arange(nf, n))):
            src, dst = sym.get(sd, f"pk_src_{grp}"), sym.get(sd, f"pk_off_{grp}")
            slots = np.concatenate([np.arange(rp[p], rp[p + 1]) for p in rows]) if len(rows) else np.array([], int)
            np.testing.assert_array_equal(np.sort(src), slots)
            places = sorted(v for c in chunks for v in c[grp + "vals"])
            np.testing.assert_array_equal(np.sort(dst), places)


def test_chunk_capacity_grows_with_the_largest_level(hs):
    """A long vertical column of fine cells in one box makes fine levels wide enough to need more
    than the smallest capacity; small boxes keep the smallest."""
    g = O.Geometry(24, 24, 16, 1, 1, 1, ov=0, near_width=0, far_mode=0)
    s = synth.grid_jacobian(g.nx, g.ny, g.nz, 13)
    big = Sym(hs, g, s).info(0)["chunk_cap"]
    g2 = O.Geometry(8, 8, 4, 2, 2, 1, ov=0, near_width=0, far_mode=0)
    s2 = synth.grid_jacobian(g2.nx, g2.ny, g2.nz, 14)
    small = Sym(hs, g2, s2).info(0)["chunk_cap"]
    assert small == CHUNK_MIN < big <= CHUNK_MAX
    g3, seed3 = WIDE
    s3 = synth.grid_jacobian(g3.nx, g3.ny, g3.nz, seed3)
    wide = Sym(hs, g3, s3)
    assert wide.info(0)["chunk_cap"] == CHUNK_MAX
    assert len(wide.get(0, "chunk_bytes")) > 2 * wide.info(0)["nlev"]   # levels split over chunks


def test_symbolic_errors_are_reported(hs):
    """A pattern that is not structurally symmetric is refused with a message, not analysed."""
    g = O.Geometry(2, 1, 2, 1, 1, 1, ov=0, near_width=0, far_mode=0)
    rp = np.array([0, 2, 3, 4, 5], dtype=np.int32)
    ci = np.array([0, 1, 1, 2, 3], dtype=np.int32)   # (0, 1) without (1, 0)
    geo = np.array([2, 1, 2, 1, 1, 1, 0, 0, 1, 1, 1, 0, 1, 1, 1], dtype=np.int32)
    err = C.create_string_buffer(256)
    h = hs.hs_create(geo.ctypes.data, 4, 5, rp.ctypes.data, ci.ctypes.data, 0, 0, 1, err, 256, 0)
    assert not h
    assert b"symmetric" in err.value


def check_pattern(hs, rp, ci):
    rp = np.ascontiguousarray(rp, dtype=np.int32)
    ci = np.ascontiguousarray(ci, dtype=np.int32)
    err = C.create_string_buffer(256)
    st = hs.hs_check_pattern(len(rp) - 1, len(ci), rp.ctypes.data, ci.ctypes.data, err, 256)
    return st, err.value.decode()


@pytest.mark.parametrize("rp,ci,msg", [
    ([0, 2, 4], [0, 1, 0, 1], ""),                                  # a valid 2-cell pattern
    ([0, 1, 2], [1, 0], "missing diagonal"),
    ([0, 2, 4], [1, 0, 0, 1], "ascending"),
    ([0, 2, 4], [0, 0, 0, 1], "ascending"),                         # a repeated column
    ([0, 2, 4], [0, 2, 0, 1], "out of range"),
    ([0, 2, 4], [0, -1, 0, 1], "out of range"),
    ([0, 2, 3], [0, 1, 1], "symmetric"),
    ([0, 2, 3], [0, 1, 0, 1], "span"),                              # row_ptr ends before col_idx
    ([1, 2, 4], [0, 1, 0, 1], "span"),
    ([0, 3, 1, 4], [0, 1, 2, 2], "monotone"),                       # a row ends past the next start
    ([0, 9, 2, 4], [0, 1, 0, 1], "monotone"),                       # a row ends past nnzb
])
def test_pattern_input_checks(hs, rp, ci, msg):
    """asm_set_matrix_bsr's checks of A's block pattern (Section 1: a structurally symmetric
    7-point pattern with diagonal blocks).  row_ptr is checked in full before col_idx is read, so a
    row that ends past nnzb is refused, not read."""
    st, err = check_pattern(hs, rp, ci)
    if not msg:
        assert st == 0 and err == ""
    else:
        assert st == 1 and msg in err, err


@pytest.mark.parametrize("name", ["cfg1", "ragged", "line"])
def test_ell_layout_is_a_bijection_onto_bsr_blocks(hs, name):
    """The ELL copy of A that the SpMV and the value fill use: block e of row r sits in slot
    e - row_ptr[r] of row r, with its column; unused slots point at the row itself (their values
    are zero)."""
    g, seed = GEOMS[name]
    s = synth.grid_jacobian(g.nx, g.ny, g.nz, seed)
    sym = Sym(hs, g, s)
    w, pad = sym.get(-1, "ell_shape")
    loc, col = sym.get(-1, "ell_loc"), sym.get(-1, "ell_col")
    n = s.n_cells
    assert pad % 64 == 0 and n <= pad < n + 64
    assert w == np.diff(s.row_ptr).max() and len(col) == w * pad
    rows = np.repeat(np.arange(n), np.diff(s.row_ptr))
    slot = np.arange(s.nnzb) - s.row_ptr[rows]
    np.testing.assert_array_equal(loc, slot * pad + rows)
    np.testing.assert_array_equal(col[loc], s.col_idx)
    used = np.zeros(w * pad, dtype=bool)
    used[loc] = True
    free = np.nonzero(~used)[0]
    r = free % pad
    np.testing.assert_array_equal(col[free], np.where(r < n, r, 0))


def expand_sum_list(g, entries):
    """cells of a sum list: cells (>= 0) and aligned 2x2x2 cell groups (~group), as a sorted array"""
    ngz, ngx = (g.nz + 1) // 2, (g.nx + 1) // 2
    out = []
    for e in entries:
        if e >= 0:
            out.append(int(e))
            continue
        G = ~int(e)
        gz, t = G % ngz, G // ngz
        gx, gy = t % ngx, t // ngx
        for y in range(2 * gy, min(2 * gy + 2, g.ny)):
            for x in range(2 * gx, min(2 * gx + 2, g.nx)):
                for z in range(2 * gz, min(2 * gz + 2, g.nz)):
                    out.append(z + g.nz * (x + g.nx * y))
    return np.sort(np.array(out, dtype=np.int64))


@pytest.mark.parametrize("name", list(GEOMS) + ["aligned"])
def test_restriction_sum_lists_cover_the_lump_cells(hs, name):
    """The lump rows' restriction (Eqs. 4.1, B.2) through the sum lists the apply reads: a near lump
    sums its list, a far lump its far box's list minus its near-region correction list, where a
    cell group stands for its cells in the grid.  Every lump must sum exactly the cells the oracle's
    local map assigns to it, each once."""
    g, seed = (O.Geometry(16, 16, 8, 2, 2, 1, ov=2), 26) if name == "aligned" else GEOMS[name]
    s = synth.grid_jacobian(g.nx, g.ny, g.nz, seed)
    sym = Sym(hs, g, s)
    pc = O.Precond(g, s.row_ptr, s.col_idx, s.vals)
    bptr, bsum = sym.get(-1, "bsum_ptr"), sym.get(-1, "bsum")
    groups_used = 0
    for sd in range(g.n_sub):
        inf = sym.info(sd)
        omap = pc.sub_map(sd)
        cid = sym.get(sd, "cidx_of_row")
        rptr, rsrc, rbox, rcorr = (sym.get(sd, k) for k in ("rptr", "rsrc", "rbox", "rcorr"))
        cptr, ccells = sym.get(sd, "corr_ptr"), sym.get(sd, "corr_cells")
        groups_used += int(np.sum(rsrc < 0) + np.sum(ccells < 0))
        for p in range(inf["nf"], inf["n"]):
            c = cid[p]
            want = np.sort(np.nonzero(omap == p)[0])
            if rbox[c] < 0:
                got = expand_sum_list(g, rsrc[rptr[c]:rptr[c + 1]])
            else:
                J = rbox[c]
                box = expand_sum_list(g, bsum[bptr[J]:bptr[J + 1]])
                assert len(np.unique(box)) == len(box)
                cut = expand_sum_list(g, ccells[cptr[rcorr[c]]:cptr[rcorr[c] + 1]]) if rcorr[c] >= 0 else []
                assert np.all(np.isin(cut, box)) and len(np.unique(cut)) == len(cut)
                got = np.setdiff1d(box, cut)
            np.testing.assert_array_equal(got, want)
    if name == "aligned":
        assert groups_used > 0 and np.sum(bsum < 0) > 0
