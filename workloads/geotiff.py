"""A reader for single-band GeoTIFF elevation grids (host-side input only).

Written from the TIFF 6.0 file layout (image file directories of tagged
fields, strips or tiles), Adobe's TIFF Technical Note 3 (the floating-point
predictor) and the GeoTIFF tags for georeferencing.  Covered: classic TIFF and
BigTIFF, either byte order; one sample per pixel of 8-64-bit unsigned or
signed integers or IEEE floats; strips or tiles; no compression or Deflate
(zlib); predictors none, horizontal differencing and floating point; the
model pixel scale with one tiepoint (a north-up grid) and GDAL's NODATA tag.
Anything else raises ValueError naming what is not supported.
"""
import struct
import zlib
from typing import Dict, List, Tuple

import numpy as np

# TIFF field types: (struct code, bytes)
_TYPES = {1: ("B", 1), 2: ("s", 1), 3: ("H", 2), 4: ("I", 4), 5: ("II", 8), 6: ("b", 1), 7: ("B", 1),
          8: ("h", 2), 9: ("i", 4), 10: ("ii", 8), 11: ("f", 4), 12: ("d", 8), 16: ("Q", 8), 17: ("q", 8),
          18: ("Q", 8)}

TAG_WIDTH, TAG_LENGTH, TAG_BITS, TAG_COMPRESSION = 256, 257, 258, 259
TAG_STRIP_OFFSETS, TAG_SAMPLES, TAG_ROWS_PER_STRIP, TAG_STRIP_BYTES = 273, 277, 278, 279
TAG_PREDICTOR = 317
TAG_TILE_WIDTH, TAG_TILE_LENGTH, TAG_TILE_OFFSETS, TAG_TILE_BYTES = 322, 323, 324, 325
TAG_SAMPLE_FORMAT = 339
TAG_PIXEL_SCALE, TAG_TIEPOINT, TAG_TRANSFORM, TAG_GEOKEYS = 33550, 33922, 34264, 34735
TAG_GDAL_NODATA = 42113
KEY_RASTER_TYPE, RASTER_PIXEL_IS_POINT = 1025, 2


def _read_ifd(data: bytes, bo: str, big: bool) -> Dict[int, List]:
    """The first image file directory: tag -> list of values."""
    if big:
        off = struct.unpack_from(bo + "Q", data, 8)[0]
        n = struct.unpack_from(bo + "Q", data, off)[0]
        first, entry, inline = off + 8, 20, 8
    else:
        off = struct.unpack_from(bo + "I", data, 4)[0]
        n = struct.unpack_from(bo + "H", data, off)[0]
        first, entry, inline = off + 2, 12, 4
    tags: Dict[int, List] = {}
    for k in range(n):
        e = first + k * entry
        if big:
            tag, typ, count = struct.unpack_from(bo + "HHQ", data, e)
            vpos = e + 12
        else:
            tag, typ, count = struct.unpack_from(bo + "HHI", data, e)
            vpos = e + 8
        if typ not in _TYPES:
            continue  # unknown field types are skipped, as TIFF readers must
        code, size = _TYPES[typ]
        nbytes = size * count
        if nbytes > inline:
            vpos = struct.unpack_from(bo + ("Q" if big else "I"), data, vpos)[0]
        raw = data[vpos:vpos + nbytes]
        if typ == 2:
            tags[tag] = [raw.split(b"\0")[0].decode("latin-1")]
        elif typ in (5, 10):
            v = struct.unpack(bo + code[0] * (2 * count), raw)
            tags[tag] = [v[2 * i] / v[2 * i + 1] for i in range(count)]
        else:
            tags[tag] = list(struct.unpack(bo + code * count, raw))
    return tags


def _dtype(bits: int, fmt: int, bo: str) -> np.dtype:
    kind = {1: "u", 2: "i", 3: "f"}.get(fmt)
    if kind is None or bits not in (8, 16, 32, 64) or (kind == "f" and bits < 32):
        raise ValueError("unsupported sample format %d with %d bits" % (fmt, bits))
    return np.dtype(("<" if bo == "<" else ">") + kind + str(bits // 8))


def _decode_block(raw: bytes, compression: int, predictor: int, dt: np.dtype, width: int, rows: int) -> np.ndarray:
    """One strip or tile as a (rows, width) array of the file's sample type."""
    if compression in (8, 32946):
        raw = zlib.decompress(raw)
    elif compression != 1:
        raise ValueError("unsupported compression %d (none and Deflate are read)" % compression)
    nb = dt.itemsize * width * rows
    buf = np.frombuffer(raw[:nb], dtype=np.uint8)
    if buf.size < nb:
        raise ValueError("a strip or tile holds fewer bytes than its pixels need")
    if predictor == 3:
        # floating point: each row holds the samples' bytes most significant
        # first (all first bytes, then all second bytes ...), differenced
        # byte by byte along the row
        b = np.cumsum(buf.reshape(rows, dt.itemsize * width), axis=1, dtype=np.uint64).astype(np.uint8)
        b = b.reshape(rows, dt.itemsize, width).transpose(0, 2, 1)
        return np.ascontiguousarray(b).view(dt.newbyteorder(">")).reshape(rows, width)
    a = buf.view(dt).reshape(rows, width)
    if predictor == 2:
        if dt.kind == "f":
            raise ValueError("horizontal differencing of floating-point samples is not defined")
        a = np.cumsum(a, axis=1, dtype=a.dtype)  # integer wraparound, as written
    elif predictor != 1:
        raise ValueError("unsupported predictor %d" % predictor)
    return a


def read_geotiff(path: str) -> Tuple[np.ndarray, float, float, float, float, np.ndarray]:
    """Read a single-band GeoTIFF of elevations.

    Returns (z, dx, dy, x0, y0, nodata) as read_esri_ascii does: z float64
    (ny, nx) with row j at y = y0 + (j + 0.5) dy (the file's first row, the
    northernmost, becomes the last); (x0, y0) the lower-left corner of the
    grid; nodata the mask of cells equal to the GDAL NODATA value (or NaN)."""
    with open(path, "rb") as f:
        data = f.read()
    if data[:2] == b"II":
        bo = "<"
    elif data[:2] == b"MM":
        bo = ">"
    else:
        raise ValueError("%s: not a TIFF file" % path)
    magic = struct.unpack_from(bo + "H", data, 2)[0]
    if magic not in (42, 43):
        raise ValueError("%s: not a TIFF file" % path)
    tags = _read_ifd(data, bo, magic == 43)

    def one(tag, default=None):
        v = tags.get(tag)
        if v is None:
            if default is None:
                raise ValueError("%s: required TIFF field %d is missing" % (path, tag))
            return default
        return v[0]

    nx, ny = int(one(TAG_WIDTH)), int(one(TAG_LENGTH))
    if int(one(TAG_SAMPLES, 1)) != 1:  # (one sample per pixel: the planar configuration does not matter)
        raise ValueError("%s: one sample per pixel is read (a single-band grid)" % path)
    dt = _dtype(int(one(TAG_BITS, 1)), int(one(TAG_SAMPLE_FORMAT, 1)), bo)
    compression, predictor = int(one(TAG_COMPRESSION, 1)), int(one(TAG_PREDICTOR, 1))
    img = np.empty((ny, nx), dtype=dt.newbyteorder("="))
    if TAG_TILE_OFFSETS in tags:
        tw, tl = int(one(TAG_TILE_WIDTH)), int(one(TAG_TILE_LENGTH))
        offs, counts = tags[TAG_TILE_OFFSETS], tags[TAG_TILE_BYTES]
        across = (nx + tw - 1) // tw
        for k, (o, c) in enumerate(zip(offs, counts)):
            tj, ti = divmod(k, across)
            blk = _decode_block(data[o:o + c], compression, predictor, dt, tw, tl)
            j0, i0 = tj * tl, ti * tw
            h, w = min(tl, ny - j0), min(tw, nx - i0)
            if h > 0 and w > 0:
                img[j0:j0 + h, i0:i0 + w] = blk[:h, :w]
    else:
        rps = int(one(TAG_ROWS_PER_STRIP, ny))
        offs, counts = tags[TAG_STRIP_OFFSETS], tags[TAG_STRIP_BYTES]
        for k, (o, c) in enumerate(zip(offs, counts)):
            j0 = k * rps
            rows = min(rps, ny - j0)
            if rows <= 0:
                break
            img[j0:j0 + rows] = _decode_block(data[o:o + c], compression, predictor, dt, nx, rows)
    z = img.astype(np.float64)

    # georeferencing: pixel scale + one tiepoint (north-up), or an axis-aligned
    # transformation matrix
    if TAG_PIXEL_SCALE in tags and TAG_TIEPOINT in tags:
        sx, sy = tags[TAG_PIXEL_SCALE][0], tags[TAG_PIXEL_SCALE][1]
        ti, tj, _, tx, ty, _ = tags[TAG_TIEPOINT][:6]
        left, top = tx - ti * sx, ty + tj * sy  # model position of raster point (0, 0)
    elif TAG_TRANSFORM in tags:
        m = tags[TAG_TRANSFORM]
        if m[1] != 0.0 or m[4] != 0.0 or not (m[5] < 0.0):
            raise ValueError("%s: only a north-up grid (no rotation) is read" % path)
        sx, sy, left, top = m[0], -m[5], m[3], m[7]
    else:
        raise ValueError("%s: no GeoTIFF pixel scale and tiepoint" % path)
    if not (sx > 0 and sy > 0):
        raise ValueError("%s: cell sizes must be positive" % path)
    keys = tags.get(TAG_GEOKEYS, [])
    for k in range(4, len(keys) - 3, 4):  # header of four shorts, then (id, location, count, value)
        if keys[k] == KEY_RASTER_TYPE and keys[k + 1] == 0 and keys[k + 3] == RASTER_PIXEL_IS_POINT:
            left, top = left - 0.5 * sx, top + 0.5 * sy  # the tiepoint named a cell centre
    x0, y0 = left, top - ny * sy

    nodata = np.isnan(z)
    if TAG_GDAL_NODATA in tags:
        text = str(tags[TAG_GDAL_NODATA][0]).strip()
        if text and text.lower() != "nan":
            nodata |= z == float(text)
    return np.ascontiguousarray(z[::-1]), float(sx), float(sy), float(x0), float(y0), np.ascontiguousarray(nodata[::-1])
