"""Host-side checks of the binding helpers (no GPU needed)."""
import numpy as np

from paper_2107_07315_gb300 import inputs as I
from paper_2107_07315_gb300 import sph


def test_packed_state_layout():
    # every field is an aligned, contiguous view with the caller's values, and
    # the fields a step changes form one leading byte range
    st, _ = I.random_state(777, seed=5, vel=0.2, stress=0.05)
    f, buf, step_bytes = sph.device_state_packed(st, device="cpu")
    base = buf.data_ptr()
    ends = []
    for k in sph.PARTICLE_KEYS:
        if st.get(k) is None:
            assert f[k] is None
            continue
        a = np.asarray(st[k])
        t = f[k]
        assert t.is_contiguous() and tuple(t.shape) == a.shape, k
        off = t.data_ptr() - base
        assert off % 256 == 0, k
        assert np.array_equal(t.numpy(), a.astype(t.numpy().dtype)), k
        ends.append((k, off, off + t.numel() * t.element_size()))
    step = [e for e in ends if e[0] in sph.STEP_KEYS]
    rest = [e for e in ends if e[0] not in sph.STEP_KEYS]
    assert max(e[2] for e in step) == step_bytes
    assert all(r[1] >= step_bytes for r in rest)
    # views alias the buffer: a write through the buffer shows in the field
    buf[f["u"].data_ptr() - base:f["u"].data_ptr() - base + 8] = 0
    assert f["u"][0].item() == 0.0


def _c_struct_fields(name):
    """Field names of `typedef struct { ... } name;` in include/sph.h, in order."""
    import os
    import re

    hdr = open(os.path.join(os.path.dirname(__file__), "..", "include", "sph.h")).read()
    m = re.search(r"typedef struct \{([^{}]*)\}\s*" + name + ";", hdr)
    assert m, name
    fields = []
    for decl in m.group(1).split(";"):
        decl = re.sub(r"/\*.*?\*/", "", decl, flags=re.S).strip()
        if not decl:
            continue
        for part in decl.split(","):
            fields.append(re.sub(r"[^A-Za-z0-9_]", " ", part).split()[-1])
    return fields


def test_ctypes_structs_match_header():
    # the binding's ctypes layouts name the C structs' fields in the same order
    # (a field appended to the header and not to the binding shifts the rest)
    for cls in (sph.sph_particles, sph.sph_eos, sph.sph_material, sph.sph_metric,
                sph.sph_external, sph.sph_rates, sph.sph_options):
        names = [f[0] for f in cls._fields_]
        assert names == _c_struct_fields(cls.__name__), cls.__name__
