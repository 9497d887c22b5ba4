"""CPU checks of the C ABI: the library builds for sm_103a, loads, exports
every entry point include/nbgs.h declares, and the ctypes structs match the
header's layout.  No compute calls (no GPU here)."""
import ctypes as C
import os
import subprocess
import textwrap

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def nb():
    from paper_1501_05810_gb300 import build
    build.build()
    from paper_1501_05810_gb300 import nbgs
    return nbgs


def test_every_declared_symbol_is_exported(nb):
    syms = nb.header_symbols()
    assert len(syms) >= 18
    for s in syms:
        assert hasattr(nb.library(), s), s
    out = subprocess.run(["nm", "-D", "--defined-only", nb.LIB_PATH], capture_output=True, text=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if l.strip()}
    assert set(syms) <= exported


def test_struct_layout_matches_header(nb, tmp_path):
    src = tmp_path / "layout.c"
    src.write_text(textwrap.dedent("""
        #include <stdio.h>
        #include <stddef.h>
        #include "nbgs.h"
        int main(void) {
            printf("%zu %zu %zu %zu %zu\\n", sizeof(nbgs_params), offsetof(nbgs_params, periodic),
                   offsetof(nbgs_params, colour_seed), offsetof(nbgs_params, contacts_per_body),
                   sizeof(nbgs_step_stats));
            printf("%zu %zu\\n", sizeof(nbgs_residuals), sizeof(nbgs_allocator));
            return 0;
        }
    """))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    a, b = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")[:2]
    got = [int(x) for x in a.split()] + [int(x) for x in b.split()]
    want = [C.sizeof(nb.nbgs_params), nb.nbgs_params.periodic.offset, nb.nbgs_params.colour_seed.offset,
            nb.nbgs_params.contacts_per_body.offset, C.sizeof(nb.nbgs_step_stats),
            C.sizeof(nb.nbgs_residuals), C.sizeof(nb.nbgs_allocator)]
    assert got == want


def test_invalid_parameters_rejected_before_any_device_work(nb):
    from paper_1501_05810_gb300 import scenes
    p = nb.make_params(scenes.default_params(dt=-1.0))
    st, h = nb.nbgs_create_scene(p, 0, None, None, None, None, None, None, None)
    assert st == nb.NBGS_EINVAL and not h.value
    p = nb.make_params(scenes.default_params(box_lo=(0, 0, 0), box_hi=(1, -1, 1)))
    st, h = nb.nbgs_create_scene(p, 0, None, None, None, None, None, None, None)
    assert st == nb.NBGS_EINVAL
    p = nb.make_params(scenes.default_params())
    p.precision = 7
    st, h = nb.nbgs_create_scene(p, 0, None, None, None, None, None, None, None)
    assert st == nb.NBGS_EINVAL
    # null scene handles are rejected
    assert nb.library().nbgs_step(None, 1, 0.0, None) == nb.NBGS_EINVAL
    assert nb.library().nbgs_sync(None) == nb.NBGS_EINVAL


def test_library_built_for_sm_103a_only(nb):
    from paper_1501_05810_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def _c_layout(tmp_path, include_dir, header, structs):
    """sizeof and every field offset of C structs, from gcc."""
    lines = []
    for cname, fields in structs:
        lines.append(f'printf("%zu\\n", sizeof({cname}));')
        lines += [f'printf("%zu\\n", offsetof({cname}, {f}));' for f in fields]
    src = tmp_path / "all_layout.c"
    src.write_text("#include <stdio.h>\n#include <stddef.h>\n#include <stdint.h>\n"
                   f'#include "{header}"\nint main(void) {{\n' + "\n".join(lines) + "\nreturn 0;\n}\n")
    exe = tmp_path / "all_layout"
    subprocess.run(["gcc", "-I", include_dir, str(src), "-o", str(exe)], check=True)
    return [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]


def _py_layout(pairs):
    out = []
    for _, cls in pairs:
        out.append(C.sizeof(cls))
        out += [getattr(cls, f).offset for f, _ in cls._fields_]
    return out


def test_every_field_of_the_binding_structs_matches_the_header(nb, tmp_path):
    pairs = [("nbgs_params", nb.nbgs_params), ("nbgs_step_stats", nb.nbgs_step_stats),
             ("nbgs_residuals", nb.nbgs_residuals), ("nbgs_batch_desc", nb.nbgs_batch_desc)]
    got = _c_layout(tmp_path, os.path.join(ROOT, "include"), "nbgs.h",
                    [(c, [f for f, _ in cls._fields_]) for c, cls in pairs])
    assert got == _py_layout(pairs)


def test_every_field_of_the_oracle_structs_matches_its_header(tmp_path):
    import oracle
    pairs = [("oracle_params", oracle.OracleParams), ("oracle_step_stats", oracle.OracleStepStats),
             ("oracle_residuals", oracle.OracleResiduals)]
    got = _c_layout(tmp_path, os.path.join(ROOT, "oracle"), "nbgs_oracle.h",
                    [(c, [f for f, _ in cls._fields_]) for c, cls in pairs])
    assert got == _py_layout(pairs)
