"""Host-side validation of the compressed-batch container and of the
checkpoint headers (no GPU: these paths copy nothing before the header has
been accepted).

The container blob is written here from the format alone (struct packing of
the documented header, sections at 16-byte aligned offsets), so that the
library's reader is checked against an independent writer; then every kind of
damage (truncation, magic, version, counts, section table, total size) must
give AEQC_ECORRUPT, never a crash or an accepted header."""
import ctypes as C
import struct

import pytest

from paper_2212_10733_gb300 import aeqc

HDR = struct.Struct("<8sII q iiii q Q 8Q 8Q Q")  # 192 bytes
assert HDR.size == 192


@pytest.fixture(scope="module")
def lib():
    from paper_2212_10733_gb300 import build
    build.build()
    return aeqc.load()


def section_lens(n, P, L, dt, outl):
    esz = 2 if dt == aeqc.DTYPE_BF16 else 4
    return [n * L * esz, n * 8, n * P * 2, n * 32, n, n * 2, outl * 8, outl * 8]


def make_blob(n=5, P=1521, L=16, dt=aeqc.DTYPE_BF16, outl=3):
    lens = section_lens(n, P, L, dt, outl)
    offs, o = [], HDR.size
    for ln in lens:
        offs.append(o)
        o = (o + ln + 15) // 16 * 16
    fields = [b"AEQCBAT1", 1, HDR.size, n, P, L, dt, 0, outl, o, *offs, *lens, 0]
    body = bytearray(o)
    body[:HDR.size] = HDR.pack(*fields)
    return bytes(body), fields


def repack(fields, total=None):
    blob = bytearray(fields[9] if total is None else total)
    blob[:HDR.size] = HDR.pack(*fields)
    return bytes(blob)


def peek(blob):
    return aeqc.batch_peek(blob)


def test_pack_size_matches_independent_layout(lib):
    for n, P, L, dt, outl in [(5, 1521, 16, aeqc.DTYPE_BF16, 3), (0, 1521, 32, aeqc.DTYPE_F32, 0),
                              (7, 100, 8, aeqc.DTYPE_F32, 700)]:
        blob, _ = make_blob(n, P, L, dt, outl)
        assert lib.aeqc_batch_pack_size(n, P, L, dt, outl) == len(blob)
    assert lib.aeqc_batch_pack_size(-1, 1521, 16, 0, 0) == 0


def test_valid_header_is_accepted(lib):
    blob, _ = make_blob()
    assert peek(blob) == dict(n=5, P=1521, L=16, latent_dtype=aeqc.DTYPE_BF16, outliers=3)
    empty, _ = make_blob(n=0, outl=0)
    assert peek(empty)["n"] == 0


def corrupt_cases():
    blob, f = make_blob()
    yield "empty", b""
    yield "short header", blob[:100]
    yield "truncated body", blob[:-16]
    yield "extra bytes", blob + b"\0" * 16
    g = list(f); g[0] = b"AEQCBAT2"; yield "magic", repack(g)
    g = list(f); g[1] = 2; yield "version", repack(g)
    g = list(f); g[2] = 200; yield "header size", repack(g)
    g = list(f); g[3] = -1; yield "negative n", repack(g)
    g = list(f); g[3] = 6; yield "n disagrees with sections", repack(g)
    g = list(f); g[4] = 0; yield "P zero", repack(g)
    g = list(f); g[4] = 5000; yield "P too large", repack(g)
    g = list(f); g[6] = 7; yield "latent dtype", repack(g)
    g = list(f); g[8] = -2; yield "negative outliers", repack(g)
    g = list(f); g[8] = 5 * 1521 + 1; yield "outliers above n P", repack(g)
    g = list(f); g[9] += 16; yield "total larger than blob", repack(g, total=len(blob))
    g = list(f); g[10 + 2] = g[10 + 1]; yield "overlapping sections", repack(g)
    g = list(f); g[10 + 3] += 8; yield "unaligned section", repack(g)
    g = list(f); g[10 + 7] = g[9]; yield "section past the end", repack(g)
    g = list(f); g[18 + 4] += 1; yield "section length", repack(g)


@pytest.mark.parametrize("name,blob", list(corrupt_cases()), ids=[c[0] for c in corrupt_cases()])
def test_corrupt_container_is_rejected(lib, name, blob):
    with pytest.raises(aeqc.AeqcError) as e:
        peek(blob)
    assert e.value.code == aeqc.ECORRUPT, name


def test_unpack_rejects_before_copying(lib):
    blob, f = make_blob()
    g = list(f); g[0] = b"XXXXXXXX"
    bad = repack(g)
    out = aeqc.aeqc_compressed()  # null device pointers: must not be touched
    rc = lib.aeqc_batch_unpack(bad, len(bad), C.byref(out), None)
    assert rc == aeqc.ECORRUPT
    rc = lib.aeqc_batch_unpack(blob[:50], 50, C.byref(out), None)
    assert rc == aeqc.ECORRUPT


def model_header(P=1521, H=64, L=16, G=1, n_group=None, n_train=None):
    desc = aeqc.aeqc_model_desc(P, H, L, 1, 0, 0, G, 0)
    if n_train is None:
        n_train = P * H + H + H * L + L + H + P  # tied: W1 b1 W2 b2 b3 b4
    if n_group is None:
        n_group = n_train + 2 * P
    hdr = b"AEQCMDL1" + struct.pack("<II", 1, 64) + bytes(desc) + struct.pack("<QQ", n_group,
                                                                               n_train)
    assert len(hdr) == 64
    return hdr, n_group, n_train


@pytest.mark.parametrize("damage", ["empty", "short", "magic", "version", "size", "groups",
                                    "counts"])
def test_corrupt_model_checkpoint_is_rejected(lib, damage):
    hdr, ng, nt = model_header()
    blob = hdr + bytes(4 * (ng + 2 * nt) + 4)
    if damage == "empty":
        blob = b""
    elif damage == "short":
        blob = blob[:40]
    elif damage == "magic":
        blob = b"AEQCMDL2" + blob[8:]
    elif damage == "version":
        blob = blob[:8] + struct.pack("<I", 9) + blob[12:]
    elif damage == "size":
        blob = blob[:-4]
    elif damage == "groups":
        h2, _, _ = model_header(G=0)
        blob = h2 + blob[64:]
    elif damage == "counts":
        h2, _, _ = model_header(n_group=ng, n_train=ng + 1)
        blob = h2 + blob[64:]
    h = C.c_void_p()
    assert lib.aeqc_model_load(blob, len(blob), C.byref(h)) == aeqc.ECORRUPT
    assert not h.value


@pytest.mark.parametrize("damage", ["short", "magic", "size", "counts"])
def test_corrupt_mlp_checkpoint_is_rejected(lib, damage):
    ni, nh = 20, 64
    n_train = ni * nh + nh + nh * nh + nh + nh * 4 + 4
    n_all = n_train + 2 * ni + 8
    hdr = b"AEQCMLP1" + struct.pack("<IIiiQQ", 1, 40, ni, nh, n_all, n_train)
    blob = hdr + bytes(4 * (n_all + 2 * n_train) + 4)
    if damage == "short":
        blob = blob[:30]
    elif damage == "magic":
        blob = b"AEQCMLPX" + blob[8:]
    elif damage == "size":
        blob = blob + b"\0"
    elif damage == "counts":
        blob = b"AEQCMLP1" + struct.pack("<IIiiQQ", 1, 40, ni, nh, n_all, n_all + 1) + blob[40:]
    h = C.c_void_p()
    assert lib.aeqc_mlp_load(blob, len(blob), C.byref(h)) == aeqc.ECORRUPT
    assert not h.value
