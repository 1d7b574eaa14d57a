/* Host driver for the CPU oracle built with AddressSanitizer and
 * UndefinedBehaviorSanitizer (tests/test_loader_sanitized.py): the oracle's
 * own decoder and interpreter over the same corpus as the loader's driver
 * (u32 program bytes, u32 input count, the program, 128-byte inputs), with
 * inputs above 2^15 threads limited so that the run stays short. */
#include "../../oracle/cufz_oracle.c"

#include <stdio.h>

_Static_assert(sizeof(orc_input) == 128, "input records are 128 bytes");

int main(int argc, char** argv) {
  if (argc != 2) return 2;
  FILE* f = fopen(argv[1], "rb");
  if (!f) return 2;
  fseek(f, 0, SEEK_END);
  long size = ftell(f);
  fseek(f, 0, SEEK_SET);
  uint8_t* buf = (uint8_t*)malloc((size_t)size);
  if (!buf || fread(buf, 1, (size_t)size, f) != (size_t)size) return 2;
  fclose(f);
  orc_opts o = {256, 64, 1u << 15};
  orc_record* recs = (orc_record*)malloc(sizeof(orc_record) * 256);
  uint8_t* bitmap = (uint8_t*)malloc(65536);
  long pos = 0, programs = 0, valid = 0, ran = 0;
  while (pos + 8 <= size) {
    uint32_t plen, nin;
    memcpy(&plen, buf + pos, 4);
    memcpy(&nin, buf + pos + 4, 4);
    pos += 8;
    uint8_t* prog = (uint8_t*)malloc(plen ? plen : 1);  /* exact size */
    memcpy(prog, buf + pos, plen);
    pos += plen;
    programs++;
    int err = 0;
    void* h = orc_load(prog, plen, &err);
    if (h) valid++;
    for (uint32_t k = 0; k < nin; k++) {
      orc_input in;
      memcpy(&in, buf + pos, sizeof(in));
      pos += (long)sizeof(in);
      if (!h) continue;
      orc_result res;
      if (orc_run(h, &in, &o, &res, recs, 256, bitmap, NULL) == 0) ran++;
    }
    if (h) orc_free(h);
    free(prog);
  }
  free(recs);
  free(bitmap);
  free(buf);
  printf("programs %ld valid %ld ran %ld\n", programs, valid, ran);
  return 0;
}
