"""The binding opens libglt.so on first use only: the package's host-side
modules (tween-frame switch, proposal features) and the benchmark's oracle
legs import without mapping the CUDA library, while any use of the library
without a built libglt.so fails loudly (no GPU needed)."""
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(code):
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    return r.stdout


def test_host_modules_do_not_map_the_library():
    out = _run(
        "import sys; sys.path.insert(0, '.')\n"
        "import paper_2607_16897_gb300.tween, paper_2607_16897_gb300.proposal\n"
        "import bench, oracle, oracle.nn, synth.jobs\n"
        "print('libglt.so' in open('/proc/self/maps').read())\n")
    assert out.strip() == "False"


def test_missing_library_fails_loudly():
    out = _run(
        "import sys; sys.path.insert(0, '.')\n"
        "import paper_2607_16897_gb300 as glt\n"
        "glt.LIB_PATH = '/nonexistent/libglt.so'\n"
        "for use in (lambda: glt.Tracker(64, 48, (50, 50, 32, 24)), lambda: glt.glt_version(),\n"
        "            lambda: glt.load()):\n"
        "    try:\n"
        "        use()\n"
        "        print('no error')\n"
        "    except ImportError as e:\n"
        "        print('ImportError', 'not built' in str(e))\n")
    assert out.split("\n")[:3] == ["ImportError True"] * 3, out
