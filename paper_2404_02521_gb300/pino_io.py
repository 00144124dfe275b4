"""PINO weight file: the format pino_load reads (serialisation only).

Little-endian layout:
  8 bytes  magic b"BSPINO01"
  8 int32  in_channels, width, modes_x, modes_y, layers, proj_hidden, 0, 0
  float32  lift_w  [in_channels][width]
           lift_b  [width]
           spec_re [layers][2*modes_y][modes_x][width][width]   (row q: ky = q for q < modes_y,
           spec_im [layers][2*modes_y][modes_x][width][width]    ky = M - 2*modes_y + q else)
           pw_w    [layers][width][width]    (in, out)
           pw_b    [layers][width]
           proj1_w [width][proj_hidden]
           proj1_b [proj_hidden]
           proj2_w [proj_hidden]
           proj2_b [1]
Batch normalisation, if the network was trained with it, is folded into pw_w / pw_b before
writing (evaluation mode).
"""
from __future__ import annotations

import struct

import numpy as np

MAGIC = b"BSPINO01"


def write_weights(path, w: dict, in_channels, width, modes_x, modes_y, layers, proj_hidden):
    with open(path, "wb") as f:
        f.write(MAGIC)
        f.write(struct.pack("<8i", in_channels, width, modes_x, modes_y, layers, proj_hidden, 0, 0))
        spec = np.asarray(w["spec_w"])
        for arr in (w["lift_w"], w["lift_b"], spec.real, spec.imag, w["pw_w"], w["pw_b"],
                    w["proj1_w"], w["proj1_b"], w["proj2_w"], np.atleast_1d(w["proj2_b"])):
            f.write(np.ascontiguousarray(arr, dtype="<f4").tobytes())


def read_weights(path):
    with open(path, "rb") as f:
        data = f.read()
    if data[:8] != MAGIC:
        raise ValueError("not a PINO weight file")
    cin, width, mx, my, L, hid, _, _ = struct.unpack("<8i", data[8:40])
    shapes = [("lift_w", (cin, width)), ("lift_b", (width,)),
              ("spec_re", (L, 2 * my, mx, width, width)), ("spec_im", (L, 2 * my, mx, width, width)),
              ("pw_w", (L, width, width)), ("pw_b", (L, width)), ("proj1_w", (width, hid)),
              ("proj1_b", (hid,)), ("proj2_w", (hid,)), ("proj2_b", (1,))]
    off = 40
    w = {}
    for name, shp in shapes:
        n = int(np.prod(shp))
        w[name] = np.frombuffer(data, dtype="<f4", count=n, offset=off).reshape(shp).astype(np.float64)
        off += 4 * n
    if off != len(data):
        raise ValueError("PINO weight file has trailing bytes")
    w["spec_w"] = w.pop("spec_re") + 1j * w.pop("spec_im")
    w["proj2_b"] = float(w["proj2_b"][0])
    arch = dict(in_channels=cin, width=width, modes_x=mx, modes_y=my, layers=L, proj_hidden=hid)
    return w, arch
