"""The C ABI without a GPU: the library loads, exports every declared entry
point, and its structs have the layout the binding assumes."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INCLUDE = os.path.join(ROOT, "include")


def declared_functions():
    names = set()
    for fn in os.listdir(INCLUDE):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(INCLUDE, fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(ms_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_paper_calls():
    names = declared_functions()
    for must in ("ms_init", "ms_encrypt_pages", "ms_decrypt_pages", "ms_sync", "ms_shutdown", "ms_strerror"):
        assert must in names


BOUNDARY_CALLS = ("ms_init", "ms_encrypt_pages", "ms_decrypt_pages", "ms_sync", "ms_shutdown", "ms_strerror",
                  "ms_submit_host", "ms_poll", "ms_wait")


def comment_before(text, name):
    """The last /* ... */ block that ends before the declaration of `name`."""
    decl = re.search(r"^[a-z][^;{}()]*\b%s\s*\(" % name, text, flags=re.M)
    assert decl, name
    blocks = [m for m in re.finditer(r"/\*.*?\*/", text, flags=re.S) if m.end() <= decl.start()]
    return blocks[-1].group(0) if blocks else ""


def test_every_boundary_call_cites_its_passage():
    """Each call of the path's boundary names the section of the paper that
    defines it, or says that the paper has no counterpart."""
    text = open(os.path.join(INCLUDE, "memshield.h")).read()
    for name in BOUNDARY_CALLS:
        c = " ".join(w for w in comment_before(text, name).split() if w not in ("/*", "*", "*/"))
        assert re.search(r"Sec\. \d\.\d", c) or "paper has no counterpart" in c, (name, c)


def test_library_exports_every_declared_symbol():
    from paper_2004_09252_b300 import memshield
    missing = [n for n in declared_functions() if not hasattr(memshield.lib, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", memshield._build.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\b[TW] (ms_[a-z0-9_]+)$", out, flags=re.M))
    assert set(declared_functions()) <= exported


def test_strerror_and_defaults():
    from paper_2004_09252_b300 import memshield as m
    assert m.strerror(m.MS_OK) == "success"
    assert "timed out" in m.strerror(m.MS_ETIMEDOUT)
    assert m.strerror(-999) == "unknown error"
    cfg = m.config_default()
    assert cfg.rounds == 20 and cfg.device == -1 and cfg.domain == 0 and cfg.timeout_ms > 0


def test_null_context_is_rejected_without_gpu():
    from paper_2004_09252_b300 import memshield as m
    assert m.lib.ms_sync(None) == m.MS_ENOTINIT
    assert m.lib.ms_encrypt_pages(None, None, 0) == m.MS_ENOTINIT
    assert m.lib.ms_shutdown(None) == m.MS_OK
    assert m.lib.ms_init(None, None, None) == m.MS_EINVAL


def test_struct_layout_matches_c():
    from paper_2004_09252_b300 import memshield as m
    src = r'''
    #include <stdio.h>
    #include <stddef.h>
    #include "memshield.h"
    int main(void) {
      printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(ms_page), sizeof(ms_config),
             offsetof(ms_config, stream), offsetof(ms_config, domain),
             offsetof(ms_config, timeout_ms), offsetof(ms_config, use_stream),
             sizeof(ms_batch_config), sizeof(ms_batch_stats), sizeof(ms_tune_result),
             offsetof(ms_tune_result, queue_gbs), offsetof(ms_tune_result, tried));
      return 0;
    }'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(c, "w").write(src)
        subprocess.check_call(["gcc", "-I", INCLUDE, c, "-o", exe])
        vals = [int(v) for v in subprocess.check_output([exe]).split()]
    cfg = m.ms_config
    assert vals == [m.PAGE_DTYPE.itemsize, ctypes.sizeof(cfg), cfg.stream.offset, cfg.domain.offset,
                    cfg.timeout_ms.offset, cfg.use_stream.offset, ctypes.sizeof(m.ms_batch_config),
                    ctypes.sizeof(m.ms_batch_stats), ctypes.sizeof(m.ms_tune_result),
                    m.ms_tune_result.queue_gbs.offset, m.ms_tune_result.tried.offset]


def test_every_struct_matches_c_field_by_field():
    """Every ctypes struct of the binding has the size and the field offsets
    of its C declaration, and the entry dtypes match ms_page / ms_page_dom."""
    from paper_2004_09252_b300 import memshield as m
    structs = [(name, cls) for name, cls in vars(m).items()
               if name.startswith("ms_") and isinstance(cls, type) and issubclass(cls, ctypes.Structure)]
    lines = []
    for name, cls in structs:
        lines.append(f'printf("%zu\\n", sizeof({name}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("%zu\\n", offsetof({name}, {f}));')
    want = []
    for name, cls in structs:
        want.append(ctypes.sizeof(cls))
        want += [getattr(cls, f).offset for f, _ in cls._fields_]
    lines.append('printf("%zu\\n%zu\\n", sizeof(ms_page), sizeof(ms_page_dom));')
    lines.append('printf("%zu\\n%zu\\n", offsetof(ms_page_dom, page_id), offsetof(ms_page_dom, domain));')
    want += [m.PAGE_DTYPE.itemsize, m.PAGE_DOM_DTYPE.itemsize, m.PAGE_DOM_DTYPE.fields["page_id"][1],
             m.PAGE_DOM_DTYPE.fields["domain"][1]]
    src = ("#include <stdio.h>\n#include <stddef.h>\n#include \"memshield.h\"\nint main(void) {\n"
           + "\n".join(lines) + "\nreturn 0;\n}\n")
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(c, "w").write(src)
        subprocess.check_call(["gcc", "-I", INCLUDE, c, "-o", exe])
        got = [int(v) for v in subprocess.check_output([exe]).split()]
    assert len(structs) >= 13
    assert got == want


def test_binding_fails_loudly_without_the_library(tmp_path):
    """No CPU fallback: importing the binding where the library is not built
    (and may not be built) raises instead of running anything."""
    import shutil
    import sys
    pkg = os.path.join(ROOT, "paper_2004_09252_b300")
    dst = tmp_path / "paper_2004_09252_b300"
    dst.mkdir()
    for f in ("__init__.py", "build.py", "memshield.py"):
        shutil.copy(os.path.join(pkg, f), dst / f)
    env = dict(os.environ, MEMSHIELD_NO_BUILD="1", PYTHONPATH=str(tmp_path))
    r = subprocess.run([sys.executable, "-c", "from paper_2004_09252_b300 import memshield"], cwd=tmp_path, env=env,
                       capture_output=True, text=True, timeout=120)
    assert r.returncode != 0 and "libmemshield.so not built" in r.stderr


def test_constants_match_the_header():
    """Every constant the binding mirrors has the header's value."""
    from paper_2004_09252_b300 import memshield as m
    names = ["MS_PAGE_BYTES", "MS_BLOCKS_PER_PAGE", "MS_KEY_BYTES", "MS_OK", "MS_EINVAL", "MS_ENOTINIT",
             "MS_ENOMEM", "MS_ECUDA", "MS_ETIMEDOUT", "MS_EBUSY", "MS_ERANGE", "MS_ESTARVED", "MS_ENCRYPT",
             "MS_DECRYPT", "MS_NOALLOC_MAX_PAGES", "MS_TICKETS", "MS_BATCH_MAX_CAPACITY", "MS_FAULT_LAUNCH",
             "MS_FAULT_COPY", "MS_FAULT_GRAPH", "MS_FAULT_SERVER", "MS_SERVE_CONTINUOUS",
             "MS_SERVE_ONE_PER_LAUNCH", "MS_SERVE_ZERO_COPY"]
    src = ("#include <stdio.h>\n#include \"memshield.h\"\nint main(void) {\n"
           + "".join(f'printf("%lld\\n", (long long)({n}));\n' for n in names) + "return 0;\n}\n")
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(c, "w").write(src)
        subprocess.check_call(["gcc", "-I", INCLUDE, c, "-o", exe])
        got = [int(v) for v in subprocess.check_output([exe]).split()]
    assert got == [getattr(m, n) for n in names]
    assert len(m.PIPE_CLASSES) == 10
