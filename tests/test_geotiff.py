"""Reading GeoTIFF elevation grids (workloads.geotiff).

No TIFF library is installed here, so the files are written by the small
writer below, from the TIFF 6.0 layout (header, one image file directory of
tagged fields sorted by tag, strips or tiles), the floating-point predictor
of TIFF Technical Note 3 and the GeoTIFF tags.  What pins the reader beyond
a round trip: every byte order, offset size, block layout, compression and
predictor must give the same grid; and a GeoTIFF and an ESRI ASCII file of
the same grid must give the same scenario.
"""
import struct
import zlib

import numpy as np
import pytest

import workloads as W
from workloads.geotiff import read_geotiff

# field types: (TIFF type, struct code)
_SHORT, _LONG, _DOUBLE, _ASCII, _LONG8 = (3, "H"), (4, "I"), (12, "d"), (2, "s"), (16, "Q")


def _encode(block, predictor):
    """One strip or tile (rows x width array of the file's sample type)."""
    rows, width = block.shape
    if predictor == 2:
        d = block.copy()
        d[:, 1:] = block[:, 1:] - block[:, :-1]  # wraps in the integer type
        return d.tobytes()
    if predictor == 3:
        be = block.astype(block.dtype.newbyteorder(">"))
        b = be.view(np.uint8).reshape(rows, width, block.dtype.itemsize).transpose(0, 2, 1).reshape(rows, -1)
        d = b.copy()
        d[:, 1:] = b[:, 1:] - b[:, :-1]  # uint8: modulo 256
        return d.tobytes()
    return block.tobytes()


def write_tiff(path, z_north_first, *, bo="<", big=False, dtype="f4", rows_per_strip=None, tile=None,
               deflate=False, predictor=1, scale=(5.0, 5.0), tiepoint=(0.0, 0.0, 1000.0, 2000.0),
               transform=None, nodata=None, point=False):
    a = np.asarray(z_north_first).astype(np.dtype(dtype).newbyteorder(bo))
    ny, nx = a.shape
    blocks = []
    if tile is None:
        rps = rows_per_strip or ny
        for j0 in range(0, ny, rps):
            blocks.append(a[j0:j0 + rps])
    else:
        tw, tl = tile
        for j0 in range(0, ny, tl):
            for i0 in range(0, nx, tw):
                t = np.zeros((tl, tw), dtype=a.dtype)
                part = a[j0:j0 + tl, i0:i0 + tw]
                t[:part.shape[0], :part.shape[1]] = part
                blocks.append(t)
    raws = [_encode(np.ascontiguousarray(b), predictor) for b in blocks]
    if deflate:
        raws = [zlib.compress(r) for r in raws]
    kind = {"f": 3, "i": 2, "u": 1}[a.dtype.kind]
    head = 16 if big else 8
    offs, pos = [], head
    for r in raws:
        offs.append(pos)
        pos += len(r)
    off_t = _LONG8 if big else _LONG
    entries = {256: (_LONG, [nx]), 257: (_LONG, [ny]), 258: (_SHORT, [a.dtype.itemsize * 8]),
               259: (_SHORT, [8 if deflate else 1]), 262: (_SHORT, [1]), 277: (_SHORT, [1]),
               284: (_SHORT, [1]), 339: (_SHORT, [kind])}
    if predictor != 1:
        entries[317] = (_SHORT, [predictor])
    if tile is None:
        entries[273] = (off_t, offs)
        entries[278] = (_LONG, [rows_per_strip or ny])
        entries[279] = (off_t, [len(r) for r in raws])
    else:
        entries[322], entries[323] = (_LONG, [tile[0]]), (_LONG, [tile[1]])
        entries[324] = (off_t, offs)
        entries[325] = (off_t, [len(r) for r in raws])
    if transform is not None:
        entries[34264] = (_DOUBLE, list(transform))
    else:
        entries[33550] = (_DOUBLE, [scale[0], scale[1], 0.0])
        entries[33922] = (_DOUBLE, [tiepoint[0], tiepoint[1], 0.0, tiepoint[2], tiepoint[3], 0.0])
    entries[34735] = (_SHORT, [1, 1, 0, 1, 1025, 0, 1, 2 if point else 1])
    if nodata is not None:
        entries[42113] = (_ASCII, [nodata])
    # the directory, then the values that do not fit in an entry
    n = len(entries)
    ifd = pos
    size = (8 + 20 * n + 8) if big else (2 + 12 * n + 4)
    extra_at = ifd + size
    ifd_bytes, extra = b"", b""
    for tag in sorted(entries):
        (typ, code), vals = entries[tag]
        if typ == 2:
            raw = vals[0].encode("latin-1") + b"\0"
            count = len(raw)
        else:
            raw = struct.pack(bo + code * len(vals), *vals)
            count = len(vals)
        inline = 8 if big else 4
        if len(raw) <= inline:
            field = raw + b"\0" * (inline - len(raw))
        else:
            field = struct.pack(bo + ("Q" if big else "I"), extra_at + len(extra))
            extra += raw + (b"\0" if len(raw) % 2 else b"")
        ifd_bytes += struct.pack(bo + ("HHQ" if big else "HHI"), tag, typ, count) + field
    ifd_bytes = struct.pack(bo + ("Q" if big else "H"), n) + ifd_bytes + b"\0" * (8 if big else 4)
    mark = b"II" if bo == "<" else b"MM"
    if big:
        header = mark + struct.pack(bo + "HHHQ", 43, 8, 0, ifd)
    else:
        header = mark + struct.pack(bo + "HI", 42, ifd)
    with open(path, "wb") as f:
        f.write(header + b"".join(raws) + ifd_bytes + extra)


def _grid(ny=37, nx=53, seed=1):
    rng = np.random.default_rng(seed)
    return (-30.0 + 50.0 * rng.uniform(size=(ny, nx))).astype(np.float32)


@pytest.mark.parametrize("bo", ["<", ">"])
@pytest.mark.parametrize("big", [False, True])
@pytest.mark.parametrize("layout", [dict(rows_per_strip=5), dict(tile=(16, 16)), dict()])
@pytest.mark.parametrize("codec", [(False, 1), (True, 1), (True, 3)])
def test_every_encoding_gives_the_same_grid(tmp_path, bo, big, layout, codec):
    z = _grid()
    p = tmp_path / "g.tif"
    write_tiff(p, z, bo=bo, big=big, deflate=codec[0], predictor=codec[1], **layout)
    g, dx, dy, x0, y0, nodata = read_geotiff(str(p))
    assert np.array_equal(g, z[::-1].astype(np.float64))  # y grows with the row index
    assert (dx, dy) == (5.0, 5.0) and (x0, y0) == (1000.0, 2000.0 - 37 * 5.0)
    assert not nodata.any()


@pytest.mark.parametrize("dtype,predictor", [("f8", 3), ("f8", 1), ("i2", 2), ("i4", 2), ("u2", 2), ("u1", 1)])
def test_sample_types(tmp_path, dtype, predictor):
    rng = np.random.default_rng(4)
    z = rng.integers(-3000 if dtype[0] == "i" else 0, 200 if dtype == "u1" else 3000, size=(21, 30))
    if dtype[0] == "f":
        z = z * 0.37
    p = tmp_path / "t.tif"
    write_tiff(p, z, dtype=dtype, predictor=predictor, deflate=True, tile=(16, 16), bo=">")
    g = read_geotiff(str(p))[0]
    assert np.array_equal(g, np.asarray(z, dtype=np.dtype(dtype)).astype(np.float64)[::-1])


def test_georeferencing_forms(tmp_path):
    z = _grid(8, 6)
    a, b, c = tmp_path / "a.tif", tmp_path / "b.tif", tmp_path / "c.tif"
    # a tiepoint at raster (2, 3) locates the same grid as one at (0, 0)
    write_tiff(a, z, scale=(2.0, 4.0), tiepoint=(2.0, 3.0, 104.0, 488.0))
    # the same grid by a transformation matrix
    write_tiff(b, z, transform=(2.0, 0, 0, 100.0, 0, -4.0, 0, 500.0, 0, 0, 0, 0, 0, 0, 0, 1))
    # PixelIsPoint: the tiepoint names the centre of the first cell
    write_tiff(c, z, scale=(2.0, 4.0), tiepoint=(0.0, 0.0, 101.0, 498.0), point=True)
    for p in (a, b, c):
        _, dx, dy, x0, y0, _ = read_geotiff(str(p))
        assert (dx, dy, x0, y0) == (2.0, 4.0, 100.0, 500.0 - 8 * 4.0), p


def test_nodata_tag(tmp_path):
    z = _grid(10, 12)
    z[3, 4] = -9999.0
    z[7, 0] = np.nan
    p = tmp_path / "n.tif"
    write_tiff(p, z, nodata="-9999")
    g, *_, nodata = read_geotiff(str(p))
    assert nodata.sum() == 2 and nodata[::-1][3, 4] and nodata[::-1][7, 0]


def test_geotiff_and_esri_ascii_give_the_same_scenario(tmp_path):
    z = _grid(24, 40, seed=9).astype(np.float64)
    z[5, 7] = -9999.0
    tif, asc = tmp_path / "d.tif", tmp_path / "d.asc"
    write_tiff(tif, z, dtype="f8", predictor=3, deflate=True, tile=(16, 16), scale=(3.0, 2.0),
               tiepoint=(0.0, 0.0, 50.0, 80.0), nodata="-9999")
    with open(asc, "w") as f:
        f.write("ncols 40\nnrows 24\nxllcorner 50\nyllcorner %r\ndx 3\ndy 2\nNODATA_value -9999\n" % (80.0 - 48.0))
        for row in z:
            f.write(" ".join("%.17g" % v for v in row) + "\n")
    for kw in (dict(), dict(crop=(2, 20, 4, 36), stride=2, manning_n=0.03)):
        a, b = W.dem_scenario(str(tif), sea_level=0.5, **kw), W.dem_scenario(str(asc), sea_level=0.5, **kw)
        assert np.array_equal(a.b, b.b) and np.array_equal(a.h, b.h) and (a.dx, a.dy) == (b.dx, b.dy)
        assert a.z_ref == b.z_ref == 0.5
    ga, gb = W.read_dem(str(tif)), W.read_esri_ascii(str(asc))
    for x, y in zip(ga, gb):
        assert np.array_equal(x, y)


def test_unsupported_files_are_rejected(tmp_path):
    z = _grid(8, 8)
    p = tmp_path / "lzw.tif"
    write_tiff(p, z)
    data = bytearray(p.read_bytes())
    # rewrite the compression field's value to LZW (5)
    n = struct.unpack_from("<H", data, struct.unpack_from("<I", data, 4)[0])[0]
    ifd = struct.unpack_from("<I", data, 4)[0] + 2
    for k in range(n):
        if struct.unpack_from("<H", data, ifd + 12 * k)[0] == 259:
            struct.pack_into("<H", data, ifd + 12 * k + 8, 5)
    p.write_bytes(bytes(data))
    with pytest.raises(ValueError, match="compression 5"):
        read_geotiff(str(p))
    q = tmp_path / "not.tif"
    q.write_bytes(b"GIF89a....")
    with pytest.raises(ValueError):
        read_geotiff(str(q))
